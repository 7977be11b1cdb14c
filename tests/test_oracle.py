"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics.

Each test checks the oracle against something other than itself: a library
routine (numpy's symmetric padding, scipy's convolve2d, erf, a scalar
minimiser), a closed form, an invariant, or values worked by hand from the
paper's equations (tests/golden/).  Together they are chosen so that a dropped
term, a wrong sign, a flipped kernel or a wrong boundary fails at least one.
"""
import os

import numpy as np
import pytest
import scipy.optimize
import scipy.signal
import scipy.special

import oracle
import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rand(shape, seed, lo=-1.0, hi=1.0):
    return synth.random_field(shape, seed, lo, hi)


# --------------------------------------------------------------------------
# boundary index and the filter bank K (Eq. diffusion, "2D convolution")
# --------------------------------------------------------------------------

@pytest.mark.parametrize("n", [1, 2, 3, 7])
def test_sym_matches_numpy_symmetric_pad(n):
    pad = 3 * n + 2
    ref = np.pad(np.arange(n), pad, mode="symmetric")
    got = [oracle.sym(i, n) for i in range(-pad, n + pad)]
    assert got == list(ref)


@pytest.mark.parametrize("H,W,ks", [(5, 7, 3), (8, 8, 5), (9, 6, 7), (12, 11, 7),
                                    (3, 4, 5), (2, 9, 3)])
def test_conv_is_symmetric_pad_then_true_convolution(H, W, ks):
    """K u equals scipy's full-flip convolution of numpy's symmetric pad."""
    u = _rand((H, W), 1 + H * W)
    k = _rand((ks, ks), 2 + ks)
    r = ks // 2
    ref = scipy.signal.convolve2d(np.pad(u, r, mode="symmetric"), k, mode="valid")
    np.testing.assert_allclose(oracle.conv(u, k), ref, rtol=1e-13, atol=1e-13)


def test_conv_is_not_correlation():
    """A non-symmetric kernel distinguishes convolution from correlation."""
    u = _rand((9, 9), 3)
    k = np.zeros((3, 3))
    k[0, 0] = 1.0  # true convolution: z(y,x) = u(y+1, x+1); correlation would be u(y-1, x-1)
    z = oracle.conv(u, k)
    np.testing.assert_allclose(z[:-1, :-1], u[1:, 1:], rtol=0, atol=0)


@pytest.mark.parametrize("H,W,ks", [(5, 7, 3), (8, 8, 5), (9, 6, 7), (12, 12, 7),
                                    (3, 3, 7)])
def test_adjoint_dense_transpose(H, W, ks):
    """K^T built column by column equals the transpose of K built the same way."""
    k = _rand((ks, ks), 10 + ks)
    n = H * W
    Kd = np.empty((n, n))
    KTd = np.empty((n, n))
    for q in range(n):
        e = np.zeros(n)
        e[q] = 1.0
        Kd[:, q] = oracle.conv(e.reshape(H, W), k).ravel()
        KTd[:, q] = oracle.conv_adj(e.reshape(H, W), k).ravel()
    np.testing.assert_allclose(KTd, Kd.T, rtol=0, atol=1e-15)


@pytest.mark.parametrize("H,W,ks", [(32, 17, 7), (64, 64, 5), (20, 9, 3)])
def test_adjoint_identity(H, W, ks):
    u = _rand((H, W), 100 + H)
    v = _rand((H, W), 200 + W)
    k = _rand((ks, ks), 300 + ks)
    lhs = np.vdot(oracle.conv(u, k), v)
    rhs = np.vdot(u, oracle.conv_adj(v, k))
    assert abs(lhs - rhs) <= 1e-12 * (np.abs(u).sum() * np.abs(v).sum() / u.size)


def test_adjoint_interior_is_rotated_kernel_convolution():
    """Away from the border K^T v = k-bar * v (Eq. diffusion, rotated kernel)."""
    H = W = 24
    ks, r = 7, 3
    v = _rand((H, W), 5)
    k = _rand((ks, ks), 6)
    kbar = k[::-1, ::-1]
    ref = scipy.signal.convolve2d(v, kbar, mode="same")
    got = oracle.conv_adj(v, k)
    np.testing.assert_allclose(got[2 * r:-2 * r, 2 * r:-2 * r],
                               ref[2 * r:-2 * r, 2 * r:-2 * r], rtol=1e-13, atol=1e-13)


# --------------------------------------------------------------------------
# influence functions phi (Gaussian RBF sums) and their derivative
# --------------------------------------------------------------------------

MU0, DELTA, GAMMA = synth.RBF_MU0, synth.RBF_DELTA, synth.RBF_GAMMA


def test_rbf_is_scaled_normal_pdf():
    import scipy.stats
    z = np.linspace(-400, 400, 97)
    for j in (0, 17, 31, 62):
        mu = MU0 + DELTA * j
        ref = scipy.stats.norm.pdf(z, loc=mu, scale=GAMMA) * GAMMA * np.sqrt(2 * np.pi)
        got = np.array([oracle.rbf(x, j, MU0, DELTA, GAMMA) for x in z])
        np.testing.assert_allclose(got, ref, rtol=1e-12, atol=1e-300)


def test_phi_at_centre_single_weight():
    w = np.zeros(63)
    w[40] = 0.37
    assert oracle.phi(MU0 + DELTA * 40, w, MU0, DELTA, GAMMA)[0] == pytest.approx(0.37, abs=0)


def test_phi_sums_all_63_terms():
    """Far-apart z values see the first and last centre: no truncation."""
    w = np.ones(63)
    z = np.array([MU0, MU0 + 62 * DELTA, 0.0])
    ref = [sum(np.exp(-(x - (MU0 + DELTA * j)) ** 2 / (2 * GAMMA ** 2)) for j in range(63))
           for x in z]
    np.testing.assert_allclose(oracle.phi(z, w, MU0, DELTA, GAMMA), ref, rtol=1e-14)


def test_phi_is_derivative_of_erf_penalty():
    """rho(z) = sum_j w_j gamma sqrt(pi/2) erf((z-mu_j)/(sqrt2 gamma)), rho' = phi (Eq. foemodel)."""
    w = synth.random_field(63, 9, -0.3, 0.3)
    mu = MU0 + DELTA * np.arange(63)

    def rho(z):
        return np.sum(w * GAMMA * np.sqrt(np.pi / 2)
                      * scipy.special.erf((z - mu) / (np.sqrt(2) * GAMMA)))

    h = 1e-4
    for z in np.linspace(-330, 330, 41):
        fd = (rho(z + h) - rho(z - h)) / (2 * h)
        assert oracle.phi(z, w, MU0, DELTA, GAMMA)[0] == pytest.approx(fd, rel=1e-7, abs=1e-10)


def test_dphi_matches_finite_difference():
    w = synth.random_field(63, 11, -0.3, 0.3)
    h = 1e-4
    z = np.linspace(-330, 330, 53)
    fd = (oracle.phi(z + h, w, MU0, DELTA, GAMMA) - oracle.phi(z - h, w, MU0, DELTA, GAMMA)) / (2 * h)
    np.testing.assert_allclose(oracle.dphi(z, w, MU0, DELTA, GAMMA), fd, rtol=1e-6, atol=1e-11)


# --------------------------------------------------------------------------
# prox of the I-divergence data term (Eqs. subproblemGpoisson/subproblemGIdiv)
# --------------------------------------------------------------------------

def _golden_prox():
    rows = []
    with open(os.path.join(GOLDEN, "prox_points.txt")) as fh:
        for line in fh:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append([float(x) for x in line.split()])
    return rows


def test_prox_hand_worked_points():
    rows = _golden_prox()
    assert len(rows) >= 10
    for ut, f, lam, u, y, x in rows:
        assert oracle.prox(np.array([ut]), f, lam)[0] == pytest.approx(u, rel=1e-15, abs=1e-15)
        if not np.isnan(y):
            assert oracle.prox_du(ut, f, lam) == pytest.approx(y, rel=1e-15, abs=1e-15)
        if not np.isnan(x):
            assert oracle.prox_dlam(ut, f, lam) == pytest.approx(x, rel=1e-15, abs=1e-15)


def test_prox_minimises_its_objective():
    """u = argmin 1/2 (u - u~)^2 + lam (u^2 - 2 f^2 log u), by a scalar minimiser."""
    g = np.random.Generator(np.random.PCG64(4))
    for _ in range(40):
        ut = g.uniform(-300, 300)
        f = g.uniform(0.5, 400)
        lam = g.uniform(0.05, 3)
        obj = lambda u: 0.5 * (u - ut) ** 2 + lam * (u * u - 2 * f * f * np.log(u))
        res = scipy.optimize.minimize_scalar(obj, bounds=(1e-9, 2000), method="bounded",
                                             options={"xatol": 1e-11})
        got = oracle.prox(np.array([ut]), f, lam)[0]
        assert got == pytest.approx(res.x, rel=1e-6)
        assert obj(got) <= obj(res.x) + 1e-9 * abs(obj(res.x))


def test_prox_optimality_residual_and_positivity():
    g = np.random.Generator(np.random.PCG64(5))
    ut = g.uniform(-1e3, 1e3, 5000)
    f = g.uniform(1e-2, 1e3, 5000)
    for lam in (1e-3, 0.5, 2.5, 7.0):
        u = oracle.prox(ut, f, lam)
        a = 1 + 2 * lam
        res = a * u * u - ut * u - 2 * lam * f * f
        scale = a * u * u + np.abs(ut * u) + 2 * lam * f * f
        assert np.all(np.abs(res) <= 1e-13 * scale)
        assert np.all(u > 0)  # positive whenever f > 0 (Sec. 3.1)


def test_prox_limits():
    ut = np.linspace(-50, 50, 101)
    np.testing.assert_array_equal(oracle.prox(ut, 3.0, 0.0), np.maximum(ut, 0.0))
    np.testing.assert_allclose(oracle.prox(ut, 0.0, 1.5), np.maximum(ut, 0.0) / 4.0, rtol=1e-15)


def test_prox_derivatives_match_finite_differences():
    g = np.random.Generator(np.random.PCG64(6))
    for _ in range(60):
        ut, f, lam = g.uniform(-200, 200), g.uniform(0.5, 300), g.uniform(0.1, 3)
        h = 1e-5 * max(1.0, abs(ut))
        fdu = (oracle.prox(np.array([ut + h]), f, lam)[0]
               - oracle.prox(np.array([ut - h]), f, lam)[0]) / (2 * h)
        assert oracle.prox_du(ut, f, lam) == pytest.approx(fdu, rel=1e-7, abs=1e-12)
        hl = 1e-6 * lam
        fdl = (oracle.prox(np.array([ut]), f, lam + hl)[0]
               - oracle.prox(np.array([ut]), f, lam - hl)[0]) / (2 * hl)
        assert oracle.prox_dlam(ut, f, lam) == pytest.approx(fdl, rel=1e-6, abs=1e-9)


# --------------------------------------------------------------------------
# the stage and the cascade
# --------------------------------------------------------------------------

def _small_model(T=2, ks=3, nk=4, seed=7):
    return synth.params(T, ks, nk, seed)


def test_zero_weights_reduce_to_scalar_prox_iterations():
    """All RBF weights 0: phi = 0, each stage is the data-term prox alone."""
    p = _small_model(T=4, ks=5, nk=3)
    p.rbf_w[:] = 0.0
    _, f = synth.single_image(13, 17, 1, cfg=90)
    u = f.copy()
    for t in range(p.T):
        u = np.array([oracle.prox(np.array([a]), b, p.lam[t])[0]
                      for a, b in zip(u.ravel(), f.ravel())]).reshape(f.shape)
    np.testing.assert_allclose(oracle.forward(f, p)[-1], u, rtol=1e-15, atol=0)


def test_constant_image_interior_follows_scalar_recursion():
    """Zero-mean filters see no structure in a constant image: far from the
    border (>= 2r per stage) each stage is u <- prox(u)."""
    p = _small_model(T=3, ks=5, nk=6, seed=8)
    c = 37.5
    H = W = 40
    f = np.full((H, W), c)
    u_all = oracle.forward(f, p)
    r = p.ks // 2
    s = c
    for t in range(p.T):
        s = oracle.prox(np.array([s]), c, p.lam[t])[0]
        m = 2 * r * (t + 1)
        np.testing.assert_allclose(u_all[t + 1][m:-m, m:-m], s, rtol=1e-12)
    # the border does feel the filters (the fold of K^T is not zero there)
    assert np.abs(u_all[1][0, :] - oracle.prox(np.array([c]), c, p.lam[0])[0]).max() > 1e-6


def test_diffusion_is_gradient_of_penalty_energy():
    """sum_i K_i^T phi_i(K_i u) = grad_u sum_i sum_p rho_i((K_i u)_p), Eq. foemodel."""
    p = _small_model(T=1, ks=5, nk=3, seed=12)
    H, W = 11, 9
    u = synth.random_field((H, W), 13, 0, 200)
    k, w = p.filters[0], p.rbf_w[0]
    mu = MU0 + DELTA * np.arange(p.nrbf)

    def energy(uu):
        e = 0.0
        for i in range(p.nk):
            z = oracle.conv(uu, k[i])[..., None]
            e += np.sum(w[i] * GAMMA * np.sqrt(np.pi / 2)
                        * scipy.special.erf((z - mu) / (np.sqrt(2) * GAMMA)))
        return e

    grad = oracle.diffusion(u, k, w, MU0, DELTA, GAMMA)
    h = 1e-3
    for (y, x) in [(0, 0), (0, 4), (1, 1), (5, 4), (10, 8), (10, 0), (3, 8), (2, 2)]:
        up, um = u.copy(), u.copy()
        up[y, x] += h
        um[y, x] -= h
        fd = (energy(up) - energy(um)) / (2 * h)
        assert grad[y, x] == pytest.approx(fd, rel=1e-6, abs=1e-9)


def test_rotation_and_transpose_equivariance():
    p = _small_model(T=2, ks=5, nk=4, seed=14)
    _, f = synth.single_image(14, 19, 1, cfg=91)
    uT = oracle.forward(f, p)[-1]
    pr = synth.Params(p.filters[:, :, ::-1, ::-1].copy(), p.rbf_w, p.lam)
    np.testing.assert_allclose(oracle.forward(f[::-1, ::-1].copy(), pr)[-1],
                               uT[::-1, ::-1], rtol=1e-12, atol=1e-12)
    pt = synth.Params(np.ascontiguousarray(p.filters.transpose(0, 1, 3, 2)), p.rbf_w, p.lam)
    np.testing.assert_allclose(oracle.forward(f.T.copy(), pt)[-1], uT.T, rtol=1e-12, atol=1e-12)


def test_stage_matches_paper_update():
    """u_t from orc_stage equals Eq. subproblemGIdiv applied to u - diffusion."""
    p = _small_model(T=1, ks=7, nk=5, seed=15)
    _, f = synth.single_image(16, 16, 2, cfg=92)
    un, ut = oracle.stage(f, f, p, 0)
    g = oracle.diffusion(f, p.filters[0], p.rbf_w[0], MU0, DELTA, GAMMA)
    np.testing.assert_allclose(ut, f - g, rtol=1e-14, atol=1e-12)
    a, lam = 1 + 2 * p.lam[0], p.lam[0]
    ref = (ut + np.sqrt(ut ** 2 + 8 * a * lam * f ** 2)) / (2 * a)
    np.testing.assert_allclose(un, ref, rtol=1e-10)


# --------------------------------------------------------------------------
# gradients (Sec. 3.2) against central finite differences of the forward
# --------------------------------------------------------------------------

def _loss(f, p, ugt):
    uT = oracle.forward(f, p)[-1]
    return 0.5 * np.sum((uT - ugt) ** 2)


def test_gradients_match_finite_differences():
    """32x32 image, 3x3x4 filters, T = 2: every filter, RBF weight and lambda
    gradient and a set of input-pixel gradients, FP64 central differences."""
    p = _small_model(T=2, ks=3, nk=4, seed=21)
    p.rbf_w *= 3.0  # larger weights make the diffusion term matter
    clean, f = synth.single_image(32, 32, 1, cfg=93)
    u_all = oracle.forward(f, p)
    eT = u_all[-1] - clean
    e0, gk, gw, gl = oracle.backward(f, p, u_all, eT)

    def check(arr, grad, hrel, name, idx_list):
        for idx in idx_list:
            old = arr[idx]
            h = hrel * max(1.0, abs(old))

            def central(hh):
                arr[idx] = old + hh
                lp = _loss(f, p, clean)
                arr[idx] = old - hh
                lm = _loss(f, p, clean)
                arr[idx] = old
                return (lp - lm) / (2 * hh)

            # Richardson extrapolation of two central differences: O(h^4)
            fd = (4.0 * central(h / 2) - central(h)) / 3.0
            g = grad[idx]
            assert abs(g - fd) <= 1e-6 * max(abs(fd), 1e-3 * gscale[name]), (name, idx, g, fd)

    gscale = {"k": np.abs(gk).max(), "w": np.abs(gw).max(), "lam": np.abs(gl).max()}
    check(p.filters, gk, 1e-4, "k", list(np.ndindex(p.filters.shape)))
    check(p.rbf_w, gw, 1e-2, "w", list(np.ndindex(p.rbf_w.shape)))
    check(p.lam, gl, 1e-4, "lam", list(np.ndindex(p.lam.shape)))

    # input pixels: corners, edges and interior (u_0 = f enters both as the
    # first state and as the data term; only the state path is dL/du_0)
    def loss_u0(u0):
        u = u0
        for t in range(p.T):
            u, _ = oracle.stage(u, f, p, t)
        return 0.5 * np.sum((u - clean) ** 2)

    pts = [(0, 0), (0, 31), (31, 0), (31, 31), (0, 15), (15, 0), (1, 1), (2, 30),
           (16, 16), (9, 23)]
    for (y, x) in pts:
        h = 1e-4 * max(1.0, abs(f[y, x]))

        def central(hh):
            up, um = f.copy(), f.copy()
            up[y, x] += hh
            um[y, x] -= hh
            return (loss_u0(up) - loss_u0(um)) / (2 * hh)

        fd = (4.0 * central(h / 2) - central(h)) / 3.0
        assert e0[y, x] == pytest.approx(fd, rel=1e-6, abs=1e-6 * np.abs(e0).max())


# --------------------------------------------------------------------------
# the other data terms: TNRD's Gaussian-denoising reaction (Sec. 2.2.1) and the
# explicit despeckling step with projection (Eq. diffusion_backP)
# --------------------------------------------------------------------------

def _energy_with_data(uu, p, f, mode):
    """E(u) = sum_i sum_p rho_i((K_i u)_p) + D(u) (Eq. foemodel), rho_i the erf
    penalty whose derivative is phi_i, D = lam/2 |u - f|^2 (Gaussian) or
    lam <log u + f^2 / (2 u^2), 1> (the data term whose gradient Eq.
    diffusion_backP subtracts)."""
    k, w, lam = p.filters[0], p.rbf_w[0], p.lam[0]
    mu = MU0 + DELTA * np.arange(p.nrbf)
    e = 0.0
    for i in range(p.nk):
        z = oracle.conv(uu, k[i])[..., None]
        e += np.sum(w[i] * GAMMA * np.sqrt(np.pi / 2)
                    * scipy.special.erf((z - mu) / (np.sqrt(2) * GAMMA)))
    if mode == 1:
        e += 0.5 * lam * np.sum((uu - f) ** 2)
    else:
        e += lam * np.sum(np.log(uu) + f ** 2 / (2 * uu ** 2))
    return e


@pytest.mark.parametrize("mode", [1, 2])
def test_explicit_stage_is_gradient_step_of_its_energy(mode):
    """u~ = u - grad E(u) with E's gradient by central differences, border
    pixels included; the Gaussian stage returns u~ itself."""
    p = _small_model(T=1, ks=5, nk=3, seed=31)
    p.dterm = mode
    H, W = 9, 11
    u = synth.random_field((H, W), 32, 40, 220)
    f = synth.random_field((H, W), 33, 30, 250)
    un, ut = oracle.stage(u, f, p, 0)
    h = 1e-3
    for (y, x) in [(0, 0), (0, 5), (1, 1), (4, 5), (8, 10), (8, 0), (3, 10), (2, 2)]:
        up, um = u.copy(), u.copy()
        up[y, x] += h
        um[y, x] -= h
        fd = (_energy_with_data(up, p, f, mode) - _energy_with_data(um, p, f, mode)) / (2 * h)
        assert u[y, x] - ut[y, x] == pytest.approx(fd, rel=1e-6, abs=1e-8)
    if mode == 1:
        np.testing.assert_array_equal(un, ut)


def test_projection_floors_at_c():
    """Eq. diffusion_backP: u_t = max(u~, c); pixels driven below c stop at c."""
    p = _small_model(T=1, ks=3, nk=4, seed=34)
    p.dterm, p.proj_c = 2, 1.0
    p.rbf_w *= 40.0                                    # a strong diffusion force
    H, W = 12, 12
    u = synth.random_field((H, W), 35, 0.5, 30)
    f = synth.random_field((H, W), 36, 0.5, 30)
    un, ut = oracle.stage(u, f, p, 0)
    below = ut < p.proj_c
    assert below.any() and (~below).any()
    np.testing.assert_array_equal(un[below], p.proj_c)
    np.testing.assert_array_equal(un[~below], ut[~below])
    # the floor moves with c
    p.proj_c = 5.0
    un5, ut5 = oracle.stage(u, f, p, 0)
    np.testing.assert_array_equal(ut5, ut)
    assert un5.min() == 5.0


@pytest.mark.parametrize("mode", [1, 2])
def test_explicit_modes_gradients_match_finite_differences(mode):
    """Every filter, RBF weight and lambda gradient and input-pixel gradients of
    the Gaussian and projection cascades (T = 2, 3x3x4, 24x24) against
    Richardson-extrapolated central differences.  Intensities are shifted to
    >= 20 so that no pixel sits at the projection's kink."""
    p = _small_model(T=2, ks=3, nk=4, seed=37)
    p.rbf_w *= 3.0
    p.dterm = mode
    p.lam = np.array([0.05, 0.1]) if mode == 1 else np.array([2.0, 3.0])
    clean, f = synth.single_image(24, 24, 8, cfg=94)
    clean, f = clean + 20.0, f + 20.0
    u_all = oracle.forward(f, p)
    for t in range(p.T):
        _, ut = oracle.stage(u_all[t], f, p, t)
        assert np.abs(ut - p.proj_c).min() > 1.0
    eT = u_all[-1] - clean
    e0, gk, gw, gl = oracle.backward(f, p, u_all, eT)
    gscale = {"k": np.abs(gk).max(), "w": np.abs(gw).max(), "lam": np.abs(gl).max()}

    def check(arr, grad, hrel, name, idx_list):
        for idx in idx_list:
            old = arr[idx]
            h = hrel * max(1.0, abs(old))

            def central(hh):
                arr[idx] = old + hh
                lp = _loss(f, p, clean)
                arr[idx] = old - hh
                lm = _loss(f, p, clean)
                arr[idx] = old
                return (lp - lm) / (2 * hh)

            fd = (4.0 * central(h / 2) - central(h)) / 3.0
            assert abs(grad[idx] - fd) <= 1e-6 * max(abs(fd), 1e-3 * gscale[name]), \
                (name, idx, grad[idx], fd)

    check(p.filters, gk, 1e-4, "k", list(np.ndindex(p.filters.shape)))
    check(p.rbf_w, gw, 1e-2, "w", list(np.ndindex(p.rbf_w.shape))[::3])
    check(p.lam, gl, 1e-4, "lam", list(np.ndindex(p.lam.shape)))

    def loss_u0(u0):
        u = u0
        for t in range(p.T):
            u, _ = oracle.stage(u, f, p, t)
        return 0.5 * np.sum((u - clean) ** 2)

    for (y, x) in [(0, 0), (0, 23), (23, 0), (23, 23), (0, 11), (12, 12), (5, 17)]:
        h = 1e-4 * max(1.0, abs(f[y, x]))

        def central(hh):
            up, um = f.copy(), f.copy()
            up[y, x] += hh
            um[y, x] -= hh
            return (loss_u0(up) - loss_u0(um)) / (2 * hh)

        fd = (4.0 * central(h / 2) - central(h)) / 3.0
        assert e0[y, x] == pytest.approx(fd, rel=1e-6, abs=1e-6 * np.abs(e0).max())
