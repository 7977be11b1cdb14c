"""Host-side checks of libtnrd.so that need no GPU: it builds, loads, exports
every symbol include/tnrd.h declares, and rejects bad arguments before it
touches the device."""
import ctypes
import os
import re

import pytest

from paper_1702_07482_gb300 import binding as B
from paper_1702_07482_gb300 import build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return B.load()


def _declared_symbols():
    syms = set()
    for name in os.listdir(os.path.join(ROOT, "include")):
        if name.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", name)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            syms |= set(re.findall(r"\b(tnrd_[a-z0-9_]+)\s*\(", txt))
    return syms


def test_exports_every_declared_symbol(lib):
    declared = _declared_symbols()
    assert "tnrd_forward" in declared and "tnrd_backward" in declared
    for s in declared:
        assert hasattr(lib, s), f"{s} declared in include/ but not exported"
    assert set(B.EXPORTS) <= declared


def test_version(lib):
    assert B.version() >= 10000


def _params(T=2, ks=7, nk=48, nrbf=63, fake=0x1000):
    p = B.tnrd_params()
    p.T, p.ksize, p.nfilt, p.nrbf = T, ks, nk, nrbf
    p.rbf_mu0, p.rbf_delta, p.rbf_gamma = -310.0, 10.0, 10.0
    p.filters = p.rbf_w = p.lambda_ = fake
    return p


def _fwd(lib, p, N=1, H=64, W=64, pitch=64, f=0x10000, u=0x200000, keep=0, algo=0,
         ws=None, wsb=0):
    return lib.tnrd_forward(ctypes.byref(p) if p is not None else None, N, H, W, pitch,
                            ctypes.c_void_p(f), ctypes.c_void_p(u), keep, algo,
                            ctypes.c_void_p(ws) if ws else None, wsb, None)


def test_argument_errors_launch_nothing(lib):
    assert _fwd(lib, None) == 1
    assert _fwd(lib, _params(ks=9, nk=80)) == 2
    assert _fwd(lib, _params(nrbf=0)) == 2
    assert _fwd(lib, _params(nrbf=65)) == 2
    p = _params()
    p.rbf_delta = 5.0  # centres closer than the width: window bound does not hold
    assert _fwd(lib, p) == 2
    assert _fwd(lib, _params(T=0)) == 1
    assert _fwd(lib, _params(), H=6) == 1          # smaller than the filter
    assert _fwd(lib, _params(), W=65, pitch=65) == 1   # pitch not a multiple of 4
    assert _fwd(lib, _params(), pitch=60) == 1     # pitch < W
    assert _fwd(lib, _params(), f=0x10004) == 1    # misaligned
    assert _fwd(lib, _params(), f=0, u=0) == 1     # null images
    assert _fwd(lib, _params(), u=0x10000 + 64) == 1   # u overlaps f
    assert _fwd(lib, _params(), algo=7) == 2
    # T >= 2 without keep_stages needs a ping-pong workspace
    assert _fwd(lib, _params(T=3), ws=None) == 5
    assert "workspace" in B.last_error()
    assert _fwd(lib, _params(), N=-1) == 1


def test_empty_batch_is_a_noop(lib):
    assert _fwd(lib, _params(), N=0, f=0, u=0) == 0


def test_workspace_sizes(lib):
    p = _params(T=5)
    # 512^2 images never take the small-image one-launch cascade
    one = 4 * 512 * 512
    assert lib.tnrd_workspace_size(0, ctypes.byref(p), 2, 512, 512, 512, 1, 0) == 0
    assert lib.tnrd_workspace_size(0, ctypes.byref(p), 2, 512, 512, 512, 0, 0) == 2 * one
    unf = lib.tnrd_workspace_size(0, ctypes.byref(p), 2, 512, 512, 512, 1, 1)
    assert unf == 2 * one * 48 + 2 * one
    assert lib.tnrd_workspace_size(0, ctypes.byref(_params(T=1)), 1, 64, 64, 64, 0, 0) == 0
    assert lib.tnrd_workspace_size(0, ctypes.byref(_params(ks=4)), 1, 64, 64, 64, 0, 0) == 0
    # small images: the ping-pong batch, plus 256 bytes for the cascade's grid-barrier
    # counter when the one-launch cascade runs (it needs a GPU to check residency)
    small = 4 * 64 * 64
    assert lib.tnrd_workspace_size(0, ctypes.byref(p), 2, 64, 64, 64, 1, 0) in (0, 256)
    assert lib.tnrd_workspace_size(0, ctypes.byref(p), 2, 64, 64, 64, 0, 0) in (2 * small,
                                                                                  2 * small + 256)


def test_plan_create_rejects_bad_batches_before_touching_the_device(lib):
    p = _params()
    pp = (B.tnrd_params * 1)(p)
    h = ctypes.c_void_p()
    img = B.tnrd_image(0x10000, 0x200000, 64, 64, 64, 0)
    arr = (B.tnrd_image * 1)(img)
    assert lib.tnrd_plan_create(ctypes.byref(h), arr, 0, pp, 1, 0, 0, None) == 1
    bad = (B.tnrd_image * 1)(B.tnrd_image(0x10000, 0x200000, 64, 64, 64, 3))
    assert lib.tnrd_plan_create(ctypes.byref(h), bad, 1, pp, 1, 0, 0, None) == 1
    small = (B.tnrd_image * 1)(B.tnrd_image(0x10000, 0x200000, 5, 64, 64, 0))
    assert lib.tnrd_plan_create(ctypes.byref(h), small, 1, pp, 1, 0, 0, None) == 1
    assert lib.tnrd_plan_create(ctypes.byref(h), arr, 1, pp, 1, 1, 0, None) == 2
    p2 = _params(T=3)
    two = (B.tnrd_params * 2)(p, p2)
    assert lib.tnrd_plan_create(ctypes.byref(h), arr, 1, two, 2, 0, 0, None) == 1
    assert not h.value


def test_forward_kernel_query_host_only():
    """tnrd_forward_kernel names a kernel for every algo without a GPU and
    rejects what tnrd_forward rejects."""
    import synth
    from paper_1702_07482_gb300 import binding as B
    from paper_1702_07482_gb300 import ops
    p = synth.params(2, 7, 48, seed=3)
    m = ops.Model.create(p.filters, p.rbf_w, p.lam, device="cpu")
    prm = m.params()
    assert B.tnrd_forward_kernel(prm, 1, 64, 64, B.ALGO["unfused"]).startswith("unf_bank_phi")
    assert "tf32" in B.tnrd_forward_kernel(prm, 1, 64, 64, B.ALGO["tf32"])
    assert "bf16" in B.tnrd_forward_kernel(prm, 1, 64, 64, B.ALGO["bf16"])
    with pytest.raises(B.TnrdError):
        B.tnrd_forward_kernel(prm, 1, 5, 64, B.ALGO["fused"])   # H < ksize


def test_data_term_validation_host_only():
    """An unknown data term, or the projection without a positive floor, is
    rejected before any launch."""
    import synth
    from paper_1702_07482_gb300 import binding as B
    from paper_1702_07482_gb300 import ops
    p = synth.params(1, 7, 48, seed=4)
    prm = ops.Model.create(p.filters, p.rbf_w, p.lam, device="cpu").params()
    for dt, c, ok in ((0, 0.0, True), (1, 0.0, True), (2, 1.0, True), (2, 0.0, False),
                      (2, float("nan"), False), (3, 1.0, False), (-1, 1.0, False)):
        prm.data_term, prm.proj_c = dt, c
        if ok:
            assert B.tnrd_forward_kernel(prm, 1, 20, 20, 0)
        else:
            with pytest.raises(B.TnrdError):
                B.tnrd_forward_kernel(prm, 1, 20, 20, 0)
