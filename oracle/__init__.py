"""Python access to the FP64 C oracle of the TRDMD stage.

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the benchmark's CPU
baseline leg may import this module; the product package never does.

`build()` compiles tnrd_oracle.c with gcc into oracle/_build/liboracle.so; the
wrappers below marshal numpy float64 arrays into the C calls (see
tnrd_oracle.h for what each computes and which equation it follows).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "tnrd_oracle.c")
_HDR = os.path.join(_HERE, "tnrd_oracle.h")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB = os.path.join(_OUT_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle (gcc, -O2, OpenMP, IEEE arithmetic: no fast-math)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(_HDR))
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= newest:
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-fopenmp",
           "-fno-fast-math", "-ffp-contract=off", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            L = ctypes.CDLL(path)
            d, i, l, P = ctypes.c_double, ctypes.c_int, ctypes.c_long, ctypes.c_void_p
            sig = {
                "orc_sym": (l, [l, l]),
                "orc_conv": (None, [P, i, i, P, i, P]),
                "orc_conv_adj": (None, [P, i, i, P, i, P]),
                "orc_rbf": (d, [d, i, d, d, d]),
                "orc_phi": (d, [d, P, i, d, d, d]),
                "orc_dphi": (d, [d, P, i, d, d, d]),
                "orc_phi_vec": (None, [P, l, P, i, d, d, d, P]),
                "orc_dphi_vec": (None, [P, l, P, i, d, d, d, P]),
                "orc_diffusion": (None, [P, i, i, P, P, i, i, i, d, d, d, P]),
                "orc_prox": (d, [d, d, d]),
                "orc_prox_vec": (None, [P, P, l, d, P]),
                "orc_prox_du": (d, [d, d, d]),
                "orc_prox_dlam": (d, [d, d, d]),
                "orc_stage": (None, [P, P, i, i, i, P, P, P, i, i, i, d, d, d, P, P]),
                "orc_forward": (None, [P, i, i, i, P, P, P, i, i, i, d, d, d, P]),
                "orc_backward": (None, [P, i, i, i, P, P, P, i, i, i, d, d, d,
                                        P, P, P, P, P, P]),
                "orc_stage_mode": (None, [P, P, i, i, i, P, P, P, i, i, i, d, d, d, i, d, P, P]),
                "orc_forward_mode": (None, [P, i, i, i, P, P, P, i, i, i, d, d, d, i, d, P]),
                "orc_backward_mode": (None, [P, i, i, i, P, P, P, i, i, i, d, d, d, i, d,
                                             P, P, P, P, P, P]),
                "orc_set_threads": (None, [i]),
                "orc_get_threads": (i, []),
            }
            for name, (res, args) in sig.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
        return _lib


def _c(a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a, a.ctypes.data_as(ctypes.c_void_p)


def sym(i: int, n: int) -> int:
    return int(lib().orc_sym(int(i), int(n)))


def conv(u, k):
    u, pu = _c(u)
    k, pk = _c(k)
    H, W = u.shape
    z = np.empty_like(u)
    lib().orc_conv(pu, H, W, pk, k.shape[0], z.ctypes.data_as(ctypes.c_void_p))
    return z


def conv_adj(v, k):
    v, pv = _c(v)
    k, pk = _c(k)
    H, W = v.shape
    out = np.empty_like(v)
    lib().orc_conv_adj(pv, H, W, pk, k.shape[0], out.ctypes.data_as(ctypes.c_void_p))
    return out


def rbf(z: float, j: int, mu0: float, delta: float, gamma: float) -> float:
    return lib().orc_rbf(float(z), int(j), mu0, delta, gamma)


def phi(z, w, mu0, delta, gamma):
    z, pz = _c(np.atleast_1d(z))
    w, pw = _c(w)
    out = np.empty_like(z)
    lib().orc_phi_vec(pz, z.size, pw, w.size, mu0, delta, gamma,
                      out.ctypes.data_as(ctypes.c_void_p))
    return out


def dphi(z, w, mu0, delta, gamma):
    z, pz = _c(np.atleast_1d(z))
    w, pw = _c(w)
    out = np.empty_like(z)
    lib().orc_dphi_vec(pz, z.size, pw, w.size, mu0, delta, gamma,
                       out.ctypes.data_as(ctypes.c_void_p))
    return out


def diffusion(u, k, w, mu0, delta, gamma):
    """sum_i K_i^T phi_i(K_i u) for one stage: k [nk][ks][ks], w [nk][nrbf]."""
    u, pu = _c(u)
    k, pk = _c(k)
    w, pw = _c(w)
    H, W = u.shape
    out = np.empty_like(u)
    lib().orc_diffusion(pu, H, W, pk, pw, k.shape[0], k.shape[1], w.shape[1],
                        mu0, delta, gamma, out.ctypes.data_as(ctypes.c_void_p))
    return out


def prox(ut, f, lam):
    ut, put = _c(ut)
    f, pf = _c(np.broadcast_to(f, ut.shape))
    out = np.empty_like(ut)
    lib().orc_prox_vec(put, pf, ut.size, float(lam), out.ctypes.data_as(ctypes.c_void_p))
    return out


def prox_du(ut: float, f: float, lam: float) -> float:
    return lib().orc_prox_du(float(ut), float(f), float(lam))


def prox_dlam(ut: float, f: float, lam: float) -> float:
    return lib().orc_prox_dlam(float(ut), float(f), float(lam))


def _pargs(p):
    k, pk = _c(p.filters)
    w, pw = _c(p.rbf_w)
    lam, pl = _c(p.lam)
    return (k, w, lam), (pk, pw, pl)


def _mode(p):
    """Data term of the model: 0 I-divergence prox (default), 1 TNRD Gaussian
    reaction, 2 explicit step with projection (floor p.proj_c)."""
    return int(getattr(p, "dterm", 0)), float(getattr(p, "proj_c", 1.0))


def stage(u_prev, f, p, t):
    """One stage (0-based t): returns (u_next, u_tilde)."""
    u_prev, pu = _c(u_prev)
    f, pf = _c(f)
    keep, (pk, pw, pl) = _pargs(p)
    H, W = u_prev.shape
    un = np.empty_like(u_prev)
    ut = np.empty_like(u_prev)
    mode, c = _mode(p)
    lib().orc_stage_mode(pu, pf, H, W, int(t), pk, pw, pl, p.nk, p.ks, p.nrbf,
                         p.mu0, p.delta, p.gamma, mode, c, un.ctypes.data_as(ctypes.c_void_p),
                         ut.ctypes.data_as(ctypes.c_void_p))
    return un, ut


def forward(f, p):
    """All stages of one image: returns u_all [T+1][H][W] (u_0 = f)."""
    f, pf = _c(f)
    keep, (pk, pw, pl) = _pargs(p)
    H, W = f.shape
    out = np.empty((p.T + 1, H, W), dtype=np.float64)
    mode, c = _mode(p)
    lib().orc_forward_mode(pf, H, W, p.T, pk, pw, pl, p.nk, p.ks, p.nrbf,
                           p.mu0, p.delta, p.gamma, mode, c, out.ctypes.data_as(ctypes.c_void_p))
    return out


def backward(f, p, u_all, e_T):
    """Gradients for one image given dL/du_T: (e_0, gk, gw, glam)."""
    f, pf = _c(f)
    keep, (pk, pw, pl) = _pargs(p)
    u_all, pua = _c(u_all)
    e_T, pe = _c(e_T)
    H, W = f.shape
    e0 = np.empty((H, W))
    gk = np.empty(p.filters.shape)
    gw = np.empty(p.rbf_w.shape)
    gl = np.empty(p.lam.shape)
    vp = lambda a: a.ctypes.data_as(ctypes.c_void_p)
    mode, c = _mode(p)
    lib().orc_backward_mode(pf, H, W, p.T, pk, pw, pl, p.nk, p.ks, p.nrbf,
                            p.mu0, p.delta, p.gamma, mode, c, pua, pe, vp(e0), vp(gk), vp(gw),
                            vp(gl))
    return e0, gk, gw, gl


def set_threads(n: int) -> None:
    lib().orc_set_threads(int(n))


def get_threads() -> int:
    return int(lib().orc_get_threads())
