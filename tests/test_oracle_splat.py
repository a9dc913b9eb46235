"""Pins for the oracle's projection, SH colour, sort and blending (Sec. 2.1, Sec. 5.1)."""
import math
import types

import numpy as np
import pytest

import oracle
from synth import scenes


def cam_identity(w=64, h=48, f=50.0, cx=None, cy=None):
    return scenes.Camera(np.concatenate([np.eye(3), np.zeros((3, 1))], axis=1),
                         float(np.float32(f)), float(np.float32(f)),
                         float(np.float32(w / 2 if cx is None else cx)),
                         float(np.float32(h / 2 if cy is None else cy)), w, h)


def one_node_asset(means, log_scales, quats=None, opacity=None, sh=None):
    n = len(means)
    quats = np.tile([1.0, 0, 0, 0], (n, 1)) if quats is None else quats
    opacity = np.full(n, 0.8) if opacity is None else opacity
    sh = np.zeros((n, 16, 3)) if sh is None else sh
    f = np.float32
    return types.SimpleNamespace(
        means=np.asarray(means, f), log_scales=np.asarray(log_scales, f), quats=np.asarray(quats, f),
        opacity=np.asarray(opacity, f), sh=np.asarray(sh, f),
        node_first=np.zeros(1, np.uint32), node_count=np.array([n], np.uint32),
        node_level=np.zeros(1, np.uint8), node_parent=np.array([-1], np.int32),
        own_sphere=np.array([[0, 0, 0, 1]], f), gaussians_per_group=256)


def project_all(asset, cam, inst=None):
    inst = inst or scenes.single_instance()
    cut = oracle.Cut(np.zeros(1, np.uint32), np.zeros(1, np.uint32), np.zeros((0, 2), np.uint32))
    return oracle.project([asset], inst, cam, cut)


# ----------------------------------------------------------------------------- projection


def test_isotropic_on_axis_closed_form():
    sigma, z, f = 0.05, 4.0, 50.0
    a = one_node_asset([[0, 0, z]], [[math.log(sigma)] * 3])
    p = project_all(a, cam_identity(f=f))
    s2 = (f * float(np.float32(sigma)) / z) ** 2
    np.testing.assert_allclose(p.cov[0], [s2, 0.0, s2], rtol=1e-6, atol=1e-12)
    np.testing.assert_allclose(p.conic[0], [1 / s2, 0.0, 1 / s2], rtol=1e-6)
    np.testing.assert_allclose(p.u[0], [32.0, 24.0])


def test_jacobian_matches_numeric_derivative():
    """Sigma_2D = J Sigma_v J^T with J the derivative of the pinhole map (inside the clamp)."""
    rng = np.random.default_rng(1)
    f = 50.0
    mu = np.array([[0.3, -0.2, 3.0], [-0.5, 0.4, 2.5], [0.1, 0.1, 6.0]])
    ls = rng.normal(-3, 0.5, (3, 3))
    q = rng.normal(size=(3, 4))
    a = one_node_asset(mu, ls, q)
    p = project_all(a, cam_identity(f=f))
    for k in range(3):
        x = a.means[k].astype(np.float64)
        eps = 1e-6
        jac = np.zeros((2, 3))
        for d in range(3):
            e = np.zeros(3)
            e[d] = eps
            hi, lo = x + e, x - e
            jac[:, d] = (np.array([f * hi[0] / hi[2], f * hi[1] / hi[2]])
                         - np.array([f * lo[0] / lo[2], f * lo[1] / lo[2]])) / (2 * eps)
        qn = a.quats[k].astype(np.float64) / np.linalg.norm(a.quats[k].astype(np.float64))
        w_, x_, y_, z_ = qn
        r = np.array([[1 - 2 * (y_ * y_ + z_ * z_), 2 * (x_ * y_ - w_ * z_), 2 * (x_ * z_ + w_ * y_)],
                      [2 * (x_ * y_ + w_ * z_), 1 - 2 * (x_ * x_ + z_ * z_), 2 * (y_ * z_ - w_ * x_)],
                      [2 * (x_ * z_ - w_ * y_), 2 * (y_ * z_ + w_ * x_), 1 - 2 * (x_ * x_ + y_ * y_)]])
        # covariance from its factor: Sigma = (R S)(R S)^T, S = diag(exp(log_scale))
        rs = r * np.exp(a.log_scales[k].astype(np.float64))[None, :]
        cov2 = jac @ (rs @ rs.T) @ jac.T
        np.testing.assert_allclose(p.cov[k], [cov2[0, 0], cov2[0, 1], cov2[1, 1]], rtol=1e-6)


def test_jacobian_clamp_outside_fov():
    sigma, z, f, w = 0.05, 4.0, 50.0, 64
    lim = 1.3 * (0.5 * w / float(np.float32(f)))
    x = 1.6 * lim * z                       # well outside the clamped cone
    a = one_node_asset([[x, 0, z]], [[math.log(sigma)] * 3])
    p = project_all(a, cam_identity(w=w, f=f))
    s2 = (f * float(np.float32(sigma)) / z) ** 2
    np.testing.assert_allclose(p.cov[0, 0], s2 * (1 + lim * lim), rtol=1e-6)
    assert p.u[0, 0] == pytest.approx(f * x / z + 32.0)


def test_isotropic_rotation_invariance():
    rng = np.random.default_rng(2)
    q = rng.normal(size=(16, 4))
    a = one_node_asset(np.tile([0.2, -0.1, 3.0], (16, 1)), np.full((16, 3), -3.0), q)
    p = project_all(a, cam_identity())
    np.testing.assert_allclose(p.cov, np.tile(p.cov[:1], (16, 1)), rtol=1e-9, atol=1e-15)


def test_instance_equals_world_gaussian():
    """Instance (s, R, t) of an asset Gaussian == the world Gaussian s R mu + t, s^2 R Sigma R^T."""
    rng = np.random.default_rng(3)
    cam = scenes.look_at((0.5, -4.0, 1.0), (0, 0, 0), 128, 96, 50.0)
    n = 12
    mu = rng.normal(0, 0.5, (n, 3))
    ls = rng.normal(-3, 0.4, (n, 3))
    q = rng.normal(size=(n, 4))
    rot = scenes.random_rotations(rng, 1)
    t = np.array([[0.2, 0.1, -0.3]])
    s = 1.7
    inst = scenes.Instances(np.zeros(1, np.uint32), rot, t, np.array([s]))
    pa = project_all(one_node_asset(mu, ls, q), cam, inst)
    mu_w = (s * (rot[0] @ mu.T)).T + t[0]
    # rotate the quaternion by R: q_w = q_R * q
    rq = _rot_to_quat(rot[0])
    qw = np.array([_qmul(rq, qq / np.linalg.norm(qq)) for qq in q])
    pw = project_all(one_node_asset(mu_w, ls + math.log(s), qw), cam)
    np.testing.assert_allclose(pa.u, pw.u, rtol=0, atol=2e-4)
    np.testing.assert_allclose(pa.cov, pw.cov, rtol=1e-4, atol=1e-9)


def _rotate_sh(sh, rot, rng):
    """SH coefficients (k, 16, 3) of the colour field d -> f(R^T d), i.e. the asset's colour field
    carried into the world frame by the rotation R.

    Band 1 by its closed form: with Y_1 = k1 (-y, z, -x), the field is k1 w . d with
    w = (-c_{1,1}, -c_{1,-1}, c_{1,0}), and f(R^T d) = k1 (R w) . d.  Bands 2 and 3 by least squares
    over random directions (each band is closed under rotation, so the fit is exact)."""
    out = np.array(sh, np.float64, copy=True)
    w = np.stack([-sh[:, 3, :], -sh[:, 1, :], sh[:, 2, :]], axis=1)       # (k, 3, channel)
    ww = np.einsum("ij,kjc->kic", rot, w)
    out[:, 3, :], out[:, 1, :], out[:, 2, :] = -ww[:, 0, :], -ww[:, 1, :], ww[:, 2, :]
    d = rng.normal(size=(400, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    y_w, y_a = oracle.sh_basis(d), oracle.sh_basis(d @ rot)               # rows: Y(d), Y(R^T d)
    for band in (slice(4, 9), slice(9, 16)):
        m, *_ = np.linalg.lstsq(y_w[:, band], y_a[:, band], rcond=None)   # Y_a = Y_w m
        out[:, band, :] = np.einsum("ij,kjc->kic", m, sh[:, band, :])
    return out


def test_instance_sh_view_direction():
    """The colour of an instanced Gaussian is evaluated along the view direction in the asset
    frame, R^T (mu_world - C) / |...|: an instance (s, R, t) with degree-1..3 SH gives the colour
    of the directly placed world Gaussian whose SH field is rotated by R.  A direction taken in
    the world frame, rotated by R instead of R^T, or without removing s and t, changes the colour
    by far more than the tolerance."""
    rng = np.random.default_rng(13)
    cam = scenes.look_at((0.7, -3.2, 1.1), (0.1, 0.2, 0.0), 128, 96, 50.0)
    n = 24
    mu = rng.normal(0, 0.5, (n, 3))
    ls = rng.normal(-3, 0.4, (n, 3))
    q = rng.normal(size=(n, 4))
    sh = rng.normal(0, 0.4, (n, 16, 3))
    rot = scenes.random_rotations(rng, 1)
    t = np.array([[0.3, -0.4, 0.2]])
    s = 1.7
    inst = scenes.Instances(np.zeros(1, np.uint32), rot, t, np.array([s]))
    pa = project_all(one_node_asset(mu, ls, q, sh=sh), cam, inst)
    sh32 = np.asarray(sh, np.float32).astype(np.float64)
    mu_w = (s * (rot[0] @ mu.astype(np.float32).astype(np.float64).T)).T + t[0]
    rq = _rot_to_quat(rot[0])
    qw = np.array([_qmul(rq, qq / np.linalg.norm(qq)) for qq in q.astype(np.float32).astype(np.float64)])
    pw = project_all(one_node_asset(mu_w, ls + math.log(s), qw, sh=_rotate_sh(sh32, rot[0], rng)), cam)
    assert pa.visible.sum() > n // 2
    np.testing.assert_allclose(pa.rgb, pw.rgb, rtol=0, atol=2e-5)
    # the test is sensitive: the same Gaussians with the unrotated SH differ clearly
    pu = project_all(one_node_asset(mu_w, ls + math.log(s), qw, sh=sh32), cam)
    assert np.abs(pa.rgb - pu.rgb).max() > 0.05


def _qmul(a, b):
    w1, x1, y1, z1 = a
    w2, x2, y2, z2 = b
    return np.array([w1 * w2 - x1 * x2 - y1 * y2 - z1 * z2, w1 * x2 + x1 * w2 + y1 * z2 - z1 * y2,
                     w1 * y2 - x1 * z2 + y1 * w2 + z1 * x2, w1 * z2 + x1 * y2 - y1 * x2 + z1 * w2])


def _rot_to_quat(r):
    w = math.sqrt(max(1.0 + r[0, 0] + r[1, 1] + r[2, 2], 1e-12)) / 2
    if w > 0.1:
        return np.array([w, (r[2, 1] - r[1, 2]) / (4 * w), (r[0, 2] - r[2, 0]) / (4 * w), (r[1, 0] - r[0, 1]) / (4 * w)])
    # fall back to an eigenvector of the rotation's symmetric 4x4 form
    k = np.array([[r[0, 0] - r[1, 1] - r[2, 2], r[1, 0] + r[0, 1], r[2, 0] + r[0, 2], r[2, 1] - r[1, 2]],
                  [r[1, 0] + r[0, 1], r[1, 1] - r[0, 0] - r[2, 2], r[2, 1] + r[1, 2], r[0, 2] - r[2, 0]],
                  [r[2, 0] + r[0, 2], r[2, 1] + r[1, 2], r[2, 2] - r[0, 0] - r[1, 1], r[1, 0] - r[0, 1]],
                  [r[2, 1] - r[1, 2], r[0, 2] - r[2, 0], r[1, 0] - r[0, 1], r[0, 0] + r[1, 1] + r[2, 2]]]) / 3
    val, vec = np.linalg.eigh(k)
    x, y, z, w = vec[:, -1]
    return np.array([w, x, y, z])


def test_culls():
    a = one_node_asset([[0, 0, 0.005], [0, 0, -1.0], [0, 0, 2.0], [30.0, 0, 2.0], [0, 0, 2.0]],
                       np.full((5, 3), -3.0), opacity=[0.8, 0.8, 0.8, 0.8, 0.003])
    p = project_all(a, cam_identity())
    # behind the near plane, behind the camera, visible, off screen, transparent
    assert p.visible.tolist() == [False, False, True, False, False]


def test_depth_key_is_rounded_depth():
    rng = np.random.default_rng(4)
    mu = rng.normal(0, 1, (200, 3)) + [0, 0, 8.0]
    a = one_node_asset(mu, np.full((200, 3), -4.0))
    p = project_all(a, cam_identity())
    z32 = p.depth_key.view(np.float32).astype(np.float64)
    # within a few float32 ulps of the exact depth, and ordered like it
    np.testing.assert_allclose(z32, a.means[:, 2].astype(np.float64), rtol=4 * 2.0 ** -24)
    assert (np.diff(p.depth_key[np.argsort(a.means[:, 2], kind="stable")].astype(np.int64)) >= 0).all()


# ----------------------------------------------------------------------------- SH


def test_sh_orthonormal_by_quadrature():
    nt, npp = 64, 128
    xg, wg = np.polynomial.legendre.leggauss(nt)       # cos(theta) nodes and weights
    phi = (np.arange(npp) + 0.5) * 2 * math.pi / npp
    ct = np.repeat(xg, npp)
    st = np.sqrt(1 - ct * ct)
    ph = np.tile(phi, nt)
    d = np.stack([st * np.cos(ph), st * np.sin(ph), ct], axis=1)
    w = np.repeat(wg, npp) * (2 * math.pi / npp)
    y = oracle.sh_basis(d)
    gram = (y * w[:, None]).T @ y
    np.testing.assert_allclose(gram, np.eye(16), atol=1e-12)


def test_sh_parity_and_degree0():
    rng = np.random.default_rng(5)
    d = rng.normal(size=(50, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    y, ym = oracle.sh_basis(d), oracle.sh_basis(-d)
    deg = np.array([0, 1, 1, 1, 2, 2, 2, 2, 2, 3, 3, 3, 3, 3, 3, 3])
    np.testing.assert_allclose(ym, y * (-1.0) ** deg[None, :], atol=1e-15)
    sh = rng.normal(0, 0.3, (50, 16, 3))
    c0 = oracle.sh_color(sh, d, degree=0)
    np.testing.assert_allclose(c0, np.maximum(0.5 + sh[:, 0, :] / (2 * math.sqrt(math.pi)), 0), rtol=1e-14)


def test_sh_degree1_is_linear_in_direction():
    # degree-1 terms are k1 * (-y, z, -x) with k1 = sqrt(3 / (4 pi))
    d = np.array([[1.0, 0, 0], [0, 1.0, 0], [0, 0, 1.0]])
    y = oracle.sh_basis(d)
    k1 = math.sqrt(3 / (4 * math.pi))
    np.testing.assert_allclose(y[:, 1:4], [[0, 0, -k1], [-k1, 0, 0], [0, k1, 0]], atol=1e-15)


# ----------------------------------------------------------------------------- blending


def test_single_gaussian_closed_form_image():
    sigma, z, f, o = 0.04, 3.0, 50.0, 0.7
    sh = np.zeros((1, 16, 3))
    sh[0, 0] = [0.4, -0.2, 0.1]
    a = one_node_asset([[0, 0, z]], [[math.log(sigma)] * 3], opacity=[o], sh=sh)
    cam = cam_identity(w=32, h=24, f=f)
    p = project_all(a, cam)
    C, T, _ = oracle.render_image(p, 32, 24)
    s = f * math.exp(float(np.float32(math.log(sigma)))) / z
    ys, xs = np.mgrid[0:24, 0:32]
    r2 = (xs + 0.5 - 16.0) ** 2 + (ys + 0.5 - 12.0) ** 2
    al = np.minimum(0.999, float(np.float32(o)) * np.exp(-r2 / (2 * s * s)))
    al = np.where(al >= 1 / 255, al, 0.0)
    col = 0.5 + sh[0, 0].astype(np.float32).astype(np.float64) * 0.5 / math.sqrt(math.pi)
    np.testing.assert_allclose(C, al[..., None] * col[None, None, :], atol=1e-12)
    np.testing.assert_allclose(T, 1 - al, atol=1e-12)


def test_two_layers_front_to_back():
    sh = np.zeros((2, 16, 3))
    sh[0, 0] = [1.0, 0, 0]
    sh[1, 0] = [0, 1.0, 0]
    # listed back first: the blend must still put the nearer one in front
    a = one_node_asset([[0, 0, 5.0], [0, 0, 3.0]], np.full((2, 3), -2.0), opacity=[0.6, 0.5], sh=sh)
    cam = cam_identity(w=16, h=16, f=40.0, cx=8.5, cy=8.5)
    p = project_all(a, cam)
    c, t, _ = oracle.render_pixels(p, [(8, 8)])
    c1 = 0.5 + np.float32(sh[1, 0]).astype(np.float64) * 0.5 / math.sqrt(math.pi)
    c0 = 0.5 + np.float32(sh[0, 0]).astype(np.float64) * 0.5 / math.sqrt(math.pi)
    a1, a0 = float(np.float32(0.5)), float(np.float32(0.6))
    np.testing.assert_allclose(c[0], a1 * c1 + (1 - a1) * a0 * c0, rtol=1e-12)
    assert t[0] == pytest.approx((1 - a1) * (1 - a0), rel=1e-12)


def test_stop_rule_identical_layers():
    n = 20
    a = one_node_asset([[0, 0, 2.0 + 0.1 * k] for k in range(n)], np.full((n, 3), -2.0),
                       opacity=np.full(n, 0.5))
    cam = cam_identity(w=16, h=16, f=40.0, cx=8.5, cy=8.5)
    p = project_all(a, cam)
    c, t, _ = oracle.render_pixels(p, [(8, 8)])
    # 0.5^13 >= 1e-4 > 0.5^14: thirteen layers are blended, the fourteenth stops the pixel
    assert t[0] == pytest.approx(2.0 ** -13, rel=1e-12)
    np.testing.assert_allclose(c[0], 0.5 * (1 - 2.0 ** -13), rtol=1e-12)


def _random_scene(seed, n=40, w=48, h=40):
    rng = np.random.default_rng(seed)
    mu = np.stack([rng.uniform(-1.2, 1.2, n), rng.uniform(-1, 1, n), rng.uniform(2.5, 6, n)], axis=1)
    a = one_node_asset(mu, rng.normal(-2.8, 0.5, (n, 3)), rng.normal(size=(n, 4)),
                       rng.uniform(0.05, 0.99, n), rng.normal(0, 0.3, (n, 16, 3)))
    cam = cam_identity(w=w, h=h, f=30.0)
    return a, cam, project_all(a, cam)


def test_pixelwise_equals_gaussianwise():
    a, cam, p = _random_scene(6)
    C, T, B = oracle.render_image(p, cam.width, cam.height)
    pix = [(x, y) for y in range(cam.height) for x in range(cam.width)]
    c, t, b = oracle.render_pixels(p, pix)
    np.testing.assert_allclose(C.reshape(-1, 3), c, rtol=0, atol=1e-13)
    np.testing.assert_allclose(T.ravel(), t, rtol=0, atol=1e-13)
    assert (B.ravel() == b).all()


def test_regions_stitch_into_the_image():
    """Tiling is only an acceleration: regions rendered on their own (each from just the Gaussians
    whose box reaches it) stitch into the whole image exactly."""
    a, cam, p = _random_scene(10, n=60, w=50, h=37)
    C, T, B = oracle.render_image(p, cam.width, cam.height)
    C2, T2, B2 = np.zeros_like(C), np.zeros_like(T), np.zeros_like(B)
    for y0 in range(0, 37, 16):
        for x0 in range(0, 50, 16):
            x1, y1 = min(x0 + 15, 49), min(y0 + 15, 36)
            near = (p.pix[:, 0] - 2 <= x1) & (p.pix[:, 1] + 2 >= x0) & (p.pix[:, 2] - 2 <= y1) & (p.pix[:, 3] + 2 >= y0)
            c, t, b = oracle.render_image(oracle.subset_projected(p, np.nonzero(near)[0]), cam.width, cam.height,
                                          region=(x0, y0, x1, y1))
            C2[y0:y1 + 1, x0:x1 + 1], T2[y0:y1 + 1, x0:x1 + 1], B2[y0:y1 + 1, x0:x1 + 1] = c, t, b
    assert np.array_equal(C, C2) and np.array_equal(T, T2) and np.array_equal(B, B2)
    assert (T < 1).sum() > 200


def test_tile_rect_covers_every_contribution():
    """Every pixel where a Gaussian reaches alpha >= 1/255 lies in a tile of its rectangle."""
    a, cam, p = _random_scene(7, n=60, w=64, h=48)
    ys, xs = np.mgrid[0:cam.height, 0:cam.width]
    for g in np.nonzero(p.visible)[0]:
        al = oracle.gaussian_alpha(p, np.full(xs.size, g), xs.ravel(), ys.ravel())
        hit = al >= 1 / 255
        tx, ty = xs.ravel()[hit] // 16, ys.ravel()[hit] // 16
        tx0, tx1, ty0, ty1 = p.rect[g]
        assert ((tx >= tx0) & (tx <= tx1) & (ty >= ty0) & (ty <= ty1)).all()
    # and an invisible Gaussian never reaches 1/255 on any pixel
    for g in np.nonzero(~p.visible & (p.depth_key.view(np.float32) > 0.01))[0]:
        if np.isfinite(p.conic[g]).all():
            al = oracle.gaussian_alpha(p, np.full(xs.size, g), xs.ravel(), ys.ravel())
            assert (al < 1 / 255).all()


def test_sorted_pairs_brute_force():
    a, cam, p = _random_scene(8, n=30, w=64, h=48)
    tiles, keys, gi, _ = oracle.sorted_pairs(p, cam)
    brute = []
    tiles_x = 4
    for g in np.nonzero(p.visible)[0]:
        tx0, tx1, ty0, ty1 = p.rect[g]
        for ty in range(ty0, ty1 + 1):
            for tx in range(tx0, tx1 + 1):
                brute.append((ty * tiles_x + tx, int(p.depth_key[g]), int(p.inst[g]), int(p.local[g])))
    brute.sort()
    got = [(int(t), int(k), int(p.inst[g]), int(p.local[g])) for t, k, g in zip(tiles, keys, gi)]
    assert got == brute


def test_sh_signs_against_complex_harmonics():
    """Y_{l,-m} = sqrt2 Im Y_l^m and Y_{l,m} = sqrt2 Re Y_l^m (m > 0), Condon-Shortley phase kept."""
    sp = pytest.importorskip("scipy.special")
    rng = np.random.default_rng(9)
    d = rng.normal(size=(40, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    theta = np.arccos(d[:, 2])
    phi = np.arctan2(d[:, 1], d[:, 0])

    def ylm(l, m):
        if hasattr(sp, "sph_harm_y"):
            return sp.sph_harm_y(l, m, theta, phi)
        return sp.sph_harm(m, l, phi, theta)

    want = []
    for l in range(4):
        for m in range(-l, l + 1):
            if m < 0:
                want.append(math.sqrt(2) * ylm(l, -m).imag)
            elif m == 0:
                want.append(ylm(l, 0).real)
            else:
                want.append(math.sqrt(2) * ylm(l, m).real)
    np.testing.assert_allclose(oracle.sh_basis(d), np.stack(want, axis=1), atol=1e-12)


def test_nodes_reaching_pixels_keeps_every_contributor(small_asset):
    """The screen bound used for sampled pixels of large frames drops no Gaussian that reaches
    alpha >= 1/255 at a sampled pixel, so the per-pixel result with and without it is identical."""
    inst = scenes.crowd_instances(60, n_assets=1, half_extent=70.0)
    cam = scenes.crowd_camera(40, 320, 180)
    cut = oracle.select([small_asset], inst, cam, 1.0)
    p = oracle.project([small_asset], inst, cam, cut)
    pix = [(x, y) for y in range(2, 180, 9) for x in range(3, 320, 11)]
    sub = oracle.nodes_reaching_pixels([small_asset], inst, cam, cut, pix)
    assert 0 < len(sub.inst) < len(cut.inst) // 2
    ps = oracle.project([small_asset], inst, cam, sub)
    kept = set((ps.inst.astype(np.int64) << 32 | ps.local.astype(np.int64)).tolist())
    vis = np.nonzero(p.visible)[0]
    n_contrib = 0
    for px, py in pix:
        al = oracle.gaussian_alpha(p, vis, px, py)
        hit = vis[al >= oracle.ALPHA_MIN]
        n_contrib += len(hit)
        g = (p.inst[hit].astype(np.int64) << 32 | p.local[hit].astype(np.int64)).tolist()
        assert kept.issuperset(g), (px, py)
    assert n_contrib > 100
    c0, t0, b0 = oracle.render_pixels(p, pix)
    c1, t1, b1 = oracle.render_pixels(ps, pix)
    assert np.array_equal(c0, c1) and np.array_equal(t0, t1) and np.array_equal(b0, b1)
    # the Gaussian-level bound on top of it keeps every contributor too, and far fewer Gaussians
    sub2, only = oracle.gaussians_reaching_pixels([small_asset], inst, cam, cut, pix)
    pg = oracle.project([small_asset], inst, cam, sub2, only=only)
    kept_g = set((pg.inst.astype(np.int64) << 32 | pg.local.astype(np.int64)).tolist())
    assert kept_g <= kept
    for px, py in pix:
        al = oracle.gaussian_alpha(p, vis, px, py)
        hit = vis[al >= oracle.ALPHA_MIN]
        assert kept_g.issuperset((p.inst[hit].astype(np.int64) << 32 | p.local[hit].astype(np.int64)).tolist())
    c2, t2, b2 = oracle.render_pixels(pg, pix)
    assert np.array_equal(c0, c2) and np.array_equal(t0, t2) and np.array_equal(b0, b2)
    # windows tested as wholes keep a superset, so the same contributors and the same pixels
    drawn = [(px, py) for (px, py), tt in zip(pix, t0) if tt < 0.99]
    wins = [(max(px - 6, 0), max(py - 6, 0), min(px + 6, 319), min(py + 6, 179)) for px, py in drawn[::max(1, len(drawn) // 3)][:3]]
    wpix = [(x, y) for x0, y0, x1, y1 in wins for y in range(y0, y1 + 1) for x in range(x0, x1 + 1)]
    sub_w, only_w = oracle.gaussians_reaching_pixels([small_asset], inst, cam, cut, wpix, windows=wins)
    sub_p, only_p = oracle.gaussians_reaching_pixels([small_asset], inst, cam, cut, wpix)
    for i, loc in only_p.items():
        assert set(loc.tolist()) <= set(only_w.get(i, np.zeros(0)).tolist())
    pw = oracle.project([small_asset], inst, cam, sub_w, only=only_w)
    cw, tw, bw = oracle.render_pixels(pw, wpix)
    cf, tf, bf = oracle.render_pixels(p, wpix)
    assert np.array_equal(cw, cf) and np.array_equal(tw, tf) and np.array_equal(bw, bf)
    assert (tf < 0.999).sum() > 50
