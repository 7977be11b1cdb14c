"""Guard bands around every buffer the library writes (in place of a memory
checker): outputs and workspaces sit inside larger canary-filled allocations
with padding columns (pitch > W) and slabs before and after; after each call
every element outside the documented output region must still hold the
canary."""
import numpy as np
import pytest
import torch

from _cases import case

pytestmark = pytest.mark.gpu

CANARY = 1234.5678
SLAB = 4096   # floats before and after each region


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1702_07482_gb300 import binding, build
    build.build()
    binding.load()


def _guarded(n, dev="cuda"):
    """A float32 region of n elements with canary slabs on both sides."""
    buf = torch.full((SLAB + n + SLAB,), CANARY, dtype=torch.float32, device=dev)
    return buf, buf[SLAB:SLAB + n]


def _check_slabs(buf, n):
    b = buf.cpu().numpy()
    assert np.all(b[:SLAB] == np.float32(CANARY)), "write before the region"
    assert np.all(b[SLAB + n:] == np.float32(CANARY)), "write after the region"


def _images(region, N, H, P):
    return region.view(N, H, P)


@pytest.mark.parametrize("algo", ["fused", "lane", "pair", "pair2", "pair4", "pair8", "unfused", "tf32",
                                  "bf16", "tf32x3"])
@pytest.mark.parametrize("keep", [0, 1])
def test_forward_writes_only_its_output(algo, keep, monkeypatch):
    if algo in ("lane", "pair", "pair2", "pair4", "pair8"):
        monkeypatch.setenv("TNRD_FUSED_KERNEL", algo)
        algo = "fused"
    from paper_1702_07482_gb300 import binding as B
    from paper_1702_07482_gb300 import ops
    H, W, P, N, T = 45, 37, 44, 2, 3
    p, f = case(H, W, 7, 48, T, N=N, cfg=200)
    m = ops.Model.create(p.filters, p.rbf_w, p.lam)
    fbuf, freg = _guarded(N * H * P)
    fimg = _images(freg, N, H, P)
    fimg[:, :, :W] = torch.tensor(f, dtype=torch.float32, device="cuda")
    nu = (T + 1) * N * H * P if keep else N * H * P
    ubuf, ureg = _guarded(nu)
    prm = m.params()
    wsb = B.tnrd_workspace_size(B.OP_FORWARD, prm, N, H, W, P, keep, B.ALGO[algo])
    wbuf, wreg = _guarded(max(1, (wsb + 3) // 4))
    stream = torch.cuda.current_stream().cuda_stream
    B.tnrd_forward(prm, N, H, W, P, fimg, ureg, keep, B.ALGO[algo], wreg if wsb else None, wsb,
                   stream)
    torch.cuda.synchronize()
    assert B.tnrd_device_status() == 0
    _check_slabs(ubuf, nu)
    _check_slabs(fbuf, N * H * P)
    _check_slabs(wbuf, max(1, (wsb + 3) // 4))
    u = ureg.view(-1, N, H, P).cpu().numpy()
    assert np.all(u[..., W:] == np.float32(CANARY)), "padding columns written"
    assert np.all(np.isfinite(u[..., :W]))
    fi = fimg.cpu().numpy()
    assert np.all(fi[..., W:] == np.float32(CANARY)), "input padding modified"


@pytest.mark.parametrize("dterm,algo", [(0, "fused"), (1, "fused"), (2, "fused"), (0, "tf32x3"),
                                        (0, "tf32"), (2, "tf32")])
def test_backward_writes_only_its_outputs(dterm, algo):
    from paper_1702_07482_gb300 import binding as B
    from paper_1702_07482_gb300 import ops
    H, W, P, N, T = 40, 33, 36, 2, 2
    p, f = case(H, W, 7, 48, T, N=N, cfg=201)
    m = ops.Model.create(p.filters, p.rbf_w, p.lam, data_term=dterm, proj_c=1.0)
    fp = torch.full((N, H, P), CANARY, device="cuda")
    fp[:, :, :W] = torch.tensor(f, dtype=torch.float32, device="cuda")
    u_all = ops.forward(m, fp, keep_stages=True, W=W)
    eT = torch.randn_like(fp)
    g0buf, g0 = _guarded(N * H * P)
    gkbuf, gk = _guarded(m.filters.numel())
    gwbuf, gw = _guarded(m.rbf_w.numel())
    glbuf, gl = _guarded(m.lam.numel())
    prm = m.params()
    wsb = B.tnrd_workspace_size(B.OP_BACKWARD, prm, N, H, W, P, 1, B.ALGO[algo])
    wbuf, wreg = _guarded((wsb + 3) // 4)
    B.tnrd_backward(prm, N, H, W, P, fp, u_all, eT, g0, gk, gw, gl, B.ALGO[algo], wreg, wsb,
                    torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    assert B.tnrd_device_status() == 0
    for buf, n in ((g0buf, N * H * P), (gkbuf, m.filters.numel()), (gwbuf, m.rbf_w.numel()),
                   (glbuf, m.lam.numel()), (wbuf, (wsb + 3) // 4)):
        _check_slabs(buf, n)
    g0i = g0.view(N, H, P).cpu().numpy()
    assert np.all(g0i[..., W:] == np.float32(CANARY))
    assert np.all(np.isfinite(g0i[..., :W]))
    assert np.all(np.isfinite(gk.cpu().numpy())) and np.all(np.isfinite(gw.cpu().numpy()))


def test_batch_and_noalloc_write_only_their_outputs():
    import synth
    from paper_1702_07482_gb300 import binding as B
    from paper_1702_07482_gb300 import ops
    p = synth.params(2, 7, 48, seed=5)
    m = ops.Model.create(p.filters, p.rbf_w, p.lam)
    sizes = [(50, 61), (33, 29), (70, 45)]
    bufs, imgs, outs = [], [], []
    for i, (H, W) in enumerate(sizes):
        P = ops.pitch_for(W) + 4
        _, f = synth.single_image(H, W, 1, 202, index=i)
        fb, fr = _guarded(H * P)
        fr.view(H, P)[:, :W] = torch.tensor(f, dtype=torch.float32, device="cuda")
        ub, ur = _guarded(H * P)
        bufs.append((fb, ub, H * P, H, W, P))
        imgs.append(B.tnrd_image(fr.data_ptr(), ur.data_ptr(), H, W, P, 0))
        outs.append(ur)
    plan = B.Plan(imgs, [m.params()])
    plan.forward(torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    assert plan.status() == 0
    for (fb, ub, n, H, W, P), ur in zip(bufs, outs):
        _check_slabs(fb, n)
        _check_slabs(ub, n)
        u = ur.view(H, P).cpu().numpy()
        assert np.all(u[:, W:] == np.float32(CANARY)) and np.all(np.isfinite(u[:, :W]))
    # the no-allocation entry point on the first image
    fb, ub, n, H, W, P = bufs[0]
    ub2, ur2 = _guarded(n)
    B.tnrd_forward_noalloc(m.params(), 1, H, W, P, fb[SLAB:SLAB + n], ur2,
                           torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    _check_slabs(ub2, n)
    assert np.all(ur2.view(H, P).cpu().numpy()[:, W:] == np.float32(CANARY))


def test_quality_writes_only_its_output():
    from paper_1702_07482_gb300 import binding as B
    H, W, P, N = 45, 37, 40, 2
    imgs = []
    for k in range(3):
        buf, reg = _guarded(N * H * P)
        v = reg.view(N, H, P)
        v[:, :, :W] = torch.rand((N, H, W), device="cuda") * 200 + 10
        imgs.append((buf, reg))
    obuf, oreg = _guarded(2 * N * 6)           # N x 6 doubles = 2 N 6 floats
    nb = B.tnrd_quality_workspace_size(N, H, W)
    wbuf, wreg = _guarded((nb + 3) // 4)
    B.tnrd_quality(imgs[0][1], imgs[1][1], imgs[2][1], N, H, W, P, 255.0, oreg, wreg, nb,
                   torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    _check_slabs(obuf, 2 * N * 6)
    _check_slabs(wbuf, (nb + 3) // 4)
    for buf, reg in imgs:
        _check_slabs(buf, N * H * P)
        assert np.all(reg.view(N, H, P).cpu().numpy()[..., W:] == np.float32(CANARY))
    assert np.all(np.isfinite(oreg.view(torch.float64).cpu().numpy()))
