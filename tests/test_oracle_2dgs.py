"""Pins of the oracle's 2DGS surfel model (Sec. 3.1, Eq. 1-3), no GPU.

(a) a face-on surfel's footprint is the closed-form isotropic Gaussian of
    std f s / z pixels, with the cutoff and alpha_min rules;
(b) the ray-plane solve: the surfel point P(u, v), taken to the camera,
    lies on the pixel's ray at depth lambda;
(c) an edge-on surfel renders nothing, and a plane met behind the camera
    counts for nothing;
(d) turning a surfel about its normal by 90 degrees with s_u, s_v swapped
    gives the same image; scaling the scene about the camera changes nothing;
(e) weights and transmittance sum to one; two stacked surfels composite
    nearest first.
"""
import math

import numpy as np

import oracle
from tests.helpers import axis_camera


def _surf(means, quats, s2, op, rgb):
    return dict(means=np.atleast_2d(means), quats=np.atleast_2d(quats), scales2=np.atleast_2d(s2),
                opacities=np.atleast_1d(op), rgb=np.atleast_2d(rgb))


def test_face_on_surfel_is_the_closed_form_gaussian():
    cam = axis_camera(W=64, H=48, fx=60.0, cx=32.5, cy=24.5)
    z, s, op = 2.0, 0.05, 0.8
    out = oracle.render_2dgs_brute(_surf([0, 0, z], [1, 0, 0, 0], [s, s], op, [1, 0, 0]), cam)
    sig = 60.0 * s / z   # 1.5 px
    for py in range(48):
        for px in range(64):
            r2 = ((px - 32) ** 2 + (py - 24) ** 2) / sig ** 2
            a = op * math.exp(-0.5 * r2)
            if r2 > 9 or a < 1 / 255:
                a = 0.0
            assert abs(out["rgb"][py, px, 0] - a) < 1e-14, (px, py)
            assert abs(out["T"][py, px] - (1 - a)) < 1e-14


def test_ray_plane_solve_lands_on_the_ray():
    g = np.random.default_rng(1)
    cam = axis_camera(W=50, H=40, fx=45.0, fy=41.0, cx=24.0, cy=21.0, t=(0.1, -0.05, 0.3))
    m = 500
    mu = g.normal(0, 0.4, (m, 3)) + [0, 0, 2.5]
    q = g.normal(size=(m, 4))
    s2 = np.exp(g.uniform(-3, -1, (m, 2)))
    px, py = g.uniform(0, 50, m), g.uniform(0, 40, m)
    r = oracle.splat_uv(mu, q, s2, cam, px, py)
    assert r["hit"].all()
    R = oracle.quat_to_rot(q)
    P = mu + (s2[:, :1] * r["u"][:, None]) * R[:, :, 0] + (s2[:, 1:] * r["v"][:, None]) * R[:, :, 1]
    w2c = np.asarray(cam["w2c"]).reshape(3, 4)
    c = P @ w2c[:, :3].T + w2c[:, 3]
    np.testing.assert_allclose(c[:, 2], r["lam"], rtol=1e-12)
    np.testing.assert_allclose(c[:, 0], r["lam"] * (px - 24.0) / 45.0, atol=1e-11)
    np.testing.assert_allclose(c[:, 1], r["lam"] * (py - 21.0) / 41.0, atol=1e-11)


def test_edge_on_surfel_renders_nothing():
    cam = axis_camera(W=32, H=32, fx=30.0, cx=16.0, cy=16.0)
    # 90 degrees about x: t_u = x, t_v = z, normal along -y; the plane holds the camera centre
    h = math.sqrt(0.5)
    out = oracle.render_2dgs_brute(_surf([0, 0, 2], [h, h, 0, 0], [0.2, 0.2], 0.9, [1, 1, 1]), cam)
    assert (out["ncontrib"] == 0).all() and (out["T"] == 1).all()


def test_turning_about_the_normal_and_scaling_the_scene():
    g = np.random.default_rng(2)
    cam = axis_camera(W=40, H=36, fx=35.0)
    n = 12
    mu = g.normal(0, 0.3, (n, 3)) + [0, 0, 2.2]
    q = g.normal(size=(n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    s2 = np.exp(g.uniform(-3, -1.8, (n, 2)))
    op = g.uniform(0.2, 0.9, n)
    rgb = g.uniform(0, 1, (n, 3))
    base = oracle.render_2dgs_brute(_surf(mu, q, s2, op, rgb), cam)
    # quaternion of a 90-degree turn about the local z (the normal): q * (cos 45, 0, 0, sin 45)
    h = math.sqrt(0.5)
    w, x, y, z = q.T
    q2 = np.stack([h * w - h * z, h * x + h * y, h * y - h * x, h * z + h * w], axis=1)
    turned = oracle.render_2dgs_brute(_surf(mu, q2, s2[:, ::-1], op, rgb), cam)
    np.testing.assert_allclose(turned["rgb"], base["rgb"], atol=1e-12)
    scaled = oracle.render_2dgs_brute(_surf(3.0 * mu, q, 3.0 * s2, op, rgb), cam)
    np.testing.assert_allclose(scaled["rgb"], base["rgb"], atol=1e-12)
    assert (base["ncontrib"] > 1).mean() > 0.05


def test_weights_sum_and_stacking_order():
    cam = axis_camera(W=32, H=32, fx=30.0, cx=16.5, cy=16.5)
    out = oracle.render_2dgs_brute(_surf([[0, 0, 2], [0.02, 0, 3]], [[1, 0, 0, 0], [1, 0, 0, 0]],
                                         [[0.1, 0.1], [0.2, 0.2]], [0.6, 0.7], [[1, 1, 1], [1, 1, 1]]), cam)
    np.testing.assert_allclose(out["rgb"][..., 0] + out["T"], 1.0, atol=1e-14)
    two = oracle.render_2dgs_brute(_surf([[0, 0, 2], [0, 0, 3]], [[1, 0, 0, 0], [1, 0, 0, 0]],
                                         [[0.1, 0.1], [0.2, 0.2]], [0.6, 0.7], [[1, 0, 0], [0, 1, 0]]), cam)
    # pixel (16, 16) is the centre of both: alpha = op there
    np.testing.assert_allclose(two["rgb"][16, 16], [0.6, 0.4 * 0.7, 0.0], atol=1e-14)


def test_plane_behind_the_camera_does_not_count():
    """A large surfel tilted almost edge-on close to the camera: for the
    lower rows its plane meets the pixel rays behind the camera (lambda < 0)
    near its centre.  Those pixels get nothing, the others do."""
    cam = axis_camera(W=32, H=32, fx=30.0, cx=16.0, cy=16.0)
    phi = math.radians(85.0)
    q = [math.cos(phi / 2), math.sin(phi / 2), 0.0, 0.0]
    surf = _surf([0, 0, 0.5], q, [5.0, 5.0], 0.9, [1, 1, 1])
    out = oracle.render_2dgs_brute(surf, cam)
    ys, xs = np.mgrid[0:32, 0:32]
    r = oracle.splat_uv(np.tile([0, 0, 0.5], (1024, 1)), np.tile(q, (1024, 1)), np.tile([5.0, 5.0], (1024, 1)), cam,
                        xs.reshape(-1) + 0.5, ys.reshape(-1) + 0.5)
    behind = (r["lam"] <= 0).reshape(32, 32)
    near_centre = ((r["u"] ** 2 + r["v"] ** 2) < 9).reshape(32, 32)
    assert (behind & near_centre).sum() > 50
    assert (out["ncontrib"][behind] == 0).all()
    assert (out["ncontrib"][~behind & near_centre] == 1).all() and (~behind & near_centre).sum() > 50


def test_surfel_rect_is_the_tight_box_of_the_projected_ellipse():
    """The dual-conic box against the projected boundary u^2 + v^2 = 9,
    sampled densely: every sample inside, every edge reached; a face-on
    surfel's box is its centre +- 3 f s / z; every pixel the render can
    touch lies inside; an ellipse reaching behind the camera gets the whole
    image."""
    g = np.random.default_rng(4)
    cam = axis_camera(W=80, H=60, fx=70.0, fy=66.0, cx=41.0, cy=29.0, t=(0.05, -0.1, 0.2))
    n = 40
    mu = g.normal(0, 0.5, (n, 3)) + [0, 0, 2.4]
    q = g.normal(size=(n, 4))
    s2 = np.exp(g.uniform(-3.5, -1.8, (n, 2)))
    r = oracle.surfel_rect(mu, q, s2, cam)
    assert r["bounded"].all()
    R = oracle.quat_to_rot(q)
    w2c = np.asarray(cam["w2c"]).reshape(3, 4)
    th = np.linspace(0, 2 * np.pi, 20001)
    for i in range(n):
        P = (mu[i][:, None] + 3 * s2[i, 0] * np.cos(th) * R[i, :, 0][:, None]
             + 3 * s2[i, 1] * np.sin(th) * R[i, :, 1][:, None])
        c = w2c[:, :3] @ P + w2c[:, 3:]
        x = 70.0 * c[0] / c[2] + 41.0
        y = 66.0 * c[1] / c[2] + 29.0
        box = r["rect"][i]
        assert x.min() >= box[0] - 1e-9 and x.max() <= box[1] + 1e-9
        assert y.min() >= box[2] - 1e-9 and y.max() <= box[3] + 1e-9
        span = max(box[1] - box[0], box[3] - box[2])
        assert abs(x.min() - box[0]) < 1e-6 * span and abs(x.max() - box[1]) < 1e-6 * span
        assert abs(y.min() - box[2]) < 1e-6 * span and abs(y.max() - box[3]) < 1e-6 * span
    # face-on
    cam0 = axis_camera(W=64, H=48, fx=60.0, cx=32.5, cy=24.5)
    f = oracle.surfel_rect([[0.1, -0.05, 2.0]], [[1, 0, 0, 0]], [[0.05, 0.08]], cam0)
    cxp, cyp = 60.0 * 0.1 / 2.0 + 32.5, 60.0 * -0.05 / 2.0 + 24.5
    np.testing.assert_allclose(f["rect"][0], [cxp - 4.5, cxp + 4.5, cyp - 7.2, cyp + 7.2], atol=1e-12)
    # the render's coverage lies inside
    ys, xs = np.mgrid[0:60, 0:80]
    for i in range(0, n, 7):
        uv = oracle.splat_uv(np.tile(mu[i], (4800, 1)), np.tile(q[i], (4800, 1)), np.tile(s2[i], (4800, 1)), cam,
                             xs.reshape(-1) + 0.5, ys.reshape(-1) + 0.5)
        inside = uv["hit"] & (uv["lam"] > 0) & (uv["u"] ** 2 + uv["v"] ** 2 <= 9)
        px, py = xs.reshape(-1)[inside] + 0.5, ys.reshape(-1)[inside] + 0.5
        box = r["rect"][i]
        assert ((px >= box[0]) & (px <= box[1]) & (py >= box[2]) & (py <= box[3])).all()
    # reaching behind the camera
    b = oracle.surfel_rect([[0, 0, 0.5]], [[1, 0, 0, 0]], [[0.5, 0.5]], cam0)
    assert b["bounded"][0] and abs(b["rect"][0][1] - b["rect"][0][0] - 2 * 3 * 60 * 0.5 / 0.5) < 1e-9
    h = math.sqrt(0.5)
    b = oracle.surfel_rect([[0, 0, 0.5]], [[h, h, 0, 0]], [[0.5, 0.5]], cam0)   # tilted: spans z = 0.5 +- 1.5
    assert not b["bounded"][0] and list(b["rect"][0]) == [0, 64, 0, 48]


def test_surfel_backward_matches_central_differences():
    g = np.random.default_rng(8)
    cam = axis_camera(W=28, H=24, fx=26.0, t=(0.03, -0.02, 0.1))
    n = 8
    q = g.normal(size=(n, 4))
    surf = dict(means=g.normal(0, 0.25, (n, 3)) + [0, 0, 2.0], quats=q / np.linalg.norm(q, axis=1, keepdims=True),
                scales2=np.exp(g.uniform(-2.6, -1.6, (n, 2))), opacities=g.uniform(0.2, 0.9, n),
                rgb=g.uniform(0, 1, (n, 3)))
    # a wide, nearly opaque surfel in front: alpha = min(0.99, op G) clamps over a few pixels
    surf["means"][0] = [0.02, -0.03, 1.6]
    surf["scales2"][0] = [0.5, 0.4]
    surf["opacities"][0] = 0.999
    surf["quats"][0] = [1.0, 0.0, 0.0, 0.0]
    prm = dict(bg=(0.2, 0.4, 0.1))
    dC = g.normal(size=(24 * 28, 3))
    grads = oracle.render_2dgs_bwd_brute(surf, cam, prm, dC)

    def loss(s):
        return float((oracle.render_2dgs_brute(s, cam, prm)["rgb"].reshape(-1, 3) * dC).sum())

    checked = 0
    for key in ("means", "quats", "scales2", "opacities", "rgb"):
        base = np.asarray(surf[key], np.float64)
        flat = base.reshape(-1)
        for i in range(flat.size):
            fds = []
            for h in (1e-6, 5e-7):
                vals = []
                for sgn in (1, -1):
                    pert = flat.copy()
                    pert[i] += sgn * h * max(1.0, abs(flat[i]))
                    vals.append(loss(dict(surf, **{key: pert.reshape(base.shape)})))
                fds.append((vals[0] - vals[1]) / (2 * h * max(1.0, abs(flat[i]))))
            if abs(fds[0] - fds[1]) > 1e-6 * max(1.0, abs(fds[0])):
                continue   # a decision flipped inside the step
            an = grads[key].reshape(-1)[i]
            assert abs(fds[0] - an) <= 2e-6 * max(1.0, abs(fds[0])), (key, i, fds[0], an)
            checked += abs(an) > 1e-8
    assert checked > 80
    uv = oracle.splat_uv(np.tile(surf["means"][0], (672, 1)), np.tile(surf["quats"][0], (672, 1)),
                         np.tile(surf["scales2"][0], (672, 1)), cam, np.tile(np.arange(28) + 0.5, 24),
                         np.repeat(np.arange(24) + 0.5, 28))
    assert (0.999 * np.exp(-0.5 * (uv["u"] ** 2 + uv["v"] ** 2)) > 0.99).sum() >= 2


def test_surfel_binning_rule_is_conservative_and_close():
    """The binary32 binning rule: every pixel the render gives a surfel's
    weight to lies in that surfel's pixel rectangle; the rectangle stays
    within the exact box widened by the rule's pad plus a pixel; tiles are
    pixel / 16; an ellipse reaching the near plane is culled."""
    g = np.random.default_rng(12)
    cam = axis_camera(W=96, H=72, fx=80.0, fy=76.0, cx=47.0, cy=37.0, t=(0.04, 0.02, 0.1))
    n = 60
    q = g.normal(size=(n, 4))
    mu = g.normal(0, 0.45, (n, 3)) + [0, 0, 2.2]
    s2 = np.exp(g.uniform(-3.5, -1.7, (n, 2)))
    b = oracle.bin_surfel_f32(mu, q, s2, cam)
    exact = oracle.surfel_rect(mu, q, s2, cam)
    ys, xs = np.mgrid[0:72, 0:96]
    kept = 0
    for i in range(n):
        if b["ntiles"][i] == 0:
            continue
        kept += 1
        x0, y0, x1, y1 = b["pix"][i]
        np.testing.assert_array_equal(b["tile"][i], [x0 // 16, y0 // 16, x1 // 16, y1 // 16])
        uv = oracle.splat_uv(np.tile(mu[i], (xs.size, 1)), np.tile(q[i], (xs.size, 1)), np.tile(s2[i], (xs.size, 1)),
                             cam, xs.reshape(-1) + 0.5, ys.reshape(-1) + 0.5)
        hit = uv["hit"] & (uv["lam"] > 0) & (uv["u"] ** 2 + uv["v"] ** 2 <= 9)
        hx, hy = xs.reshape(-1)[hit], ys.reshape(-1)[hit]
        assert ((hx >= x0) & (hx <= x1) & (hy >= y0) & (hy <= y1)).all(), i
        ex0, ex1, ey0, ey1 = exact["rect"][i]
        pad = max(ex1 - ex0, ey1 - ey0) / 64 + 0.5 + 1.0
        assert x0 >= max(0, np.floor(ex0 - pad)) and x1 <= min(95, np.ceil(ex1 + pad)), i
        assert y0 >= max(0, np.floor(ey0 - pad)) and y1 <= min(71, np.ceil(ey1 + pad)), i
        assert b["dbits"][i] != 0xFFFFFFFF
    assert kept > 40
    h = np.float32(np.sqrt(0.5))
    near = oracle.bin_surfel_f32([[0, 0, 0.6]], [[h, h, 0, 0]], [[0.2, 0.2]], cam)   # spans z = 0.7 -+ 0.6
    assert near["ntiles"][0] == 0
    # face-on: centre +- 3 f s / z, widened by the pad
    cam0 = axis_camera(W=64, H=48, fx=60.0, cx=32.0, cy=24.0)
    f = oracle.bin_surfel_f32([[0.0, 0.0, 2.0]], [[1, 0, 0, 0]], [[0.05, 0.05]], cam0)
    e = 3 * 60 * 0.05 / 2 + (2 * 4.5) / 64 + 0.5   # half-width + pad
    assert list(f["pix"][0]) == [int(np.ceil(32 - e - 0.5)), int(np.ceil(24 - e - 0.5)),
                                 int(np.floor(32 + e - 0.5)), int(np.floor(24 + e - 0.5))]


def test_tiled_surfel_render_equals_brute_force():
    g = np.random.default_rng(14)
    cam = axis_camera(W=70, H=52, fx=60.0, t=(0.02, -0.03, 0.0))
    n = 150
    q = g.normal(size=(n, 4))
    surf = dict(means=g.normal(0, 0.4, (n, 3)) + [0, 0, 2.5], quats=q, scales2=np.exp(g.uniform(-3.2, -1.9, (n, 2))),
                opacities=g.uniform(0.1, 0.95, n), rgb=g.uniform(0, 1, (n, 3)))
    surf = {k: np.asarray(v, np.float32).astype(np.float64) for k, v in surf.items()}   # binary32 inputs
    prm = dict(bg=(0.1, 0.3, 0.2))
    tiled = oracle.render_2dgs(surf, cam, prm)
    assert (tiled["bins"]["ntiles"] > 0).mean() > 0.9    # the rest lie off the image
    brute = oracle.render_2dgs_brute(surf, cam, prm)
    np.testing.assert_allclose(tiled["rgb"], brute["rgb"], atol=1e-12)
    np.testing.assert_array_equal(tiled["ncontrib"], brute["ncontrib"])
    assert (brute["ncontrib"] > 3).mean() > 0.2


def test_projective_map_gives_the_same_intersection():
    """The two-plane form through T = K [a b c] (the form a per-pixel kernel
    evaluates from a per-surfel record) equals the ray-plane solve."""
    g = np.random.default_rng(15)
    cam = axis_camera(W=60, H=50, fx=52.0, fy=49.0, cx=29.0, cy=26.0, t=(0.05, 0.02, 0.2))
    m = 2000
    mu = g.normal(0, 0.4, (m, 3)) + [0, 0, 2.3]
    q = g.normal(size=(m, 4))
    s2 = np.exp(g.uniform(-3, -1, (m, 2)))
    px, py = g.uniform(0, 60, m), g.uniform(0, 50, m)
    a = oracle.splat_uv(mu, q, s2, cam, px, py)
    b = oracle.splat_uv_T(mu, q, s2, cam, px, py)
    ok = a["hit"] & (np.abs(a["u"]) < 50) & (np.abs(a["v"]) < 50)   # away from grazing rays
    assert ok.mean() > 0.8
    np.testing.assert_allclose(b["u"][ok], a["u"][ok], rtol=1e-8, atol=1e-9)
    np.testing.assert_allclose(b["v"][ok], a["v"][ok], rtol=1e-8, atol=1e-9)
    np.testing.assert_allclose(b["depth"][ok], a["lam"][ok], rtol=1e-9)


def test_tiled_surfel_backward_equals_brute_force():
    g = np.random.default_rng(16)
    cam = axis_camera(W=52, H=44, fx=46.0, t=(0.01, 0.02, 0.0))
    n = 60
    surf = dict(means=g.normal(0, 0.35, (n, 3)) + [0, 0, 2.4], quats=g.normal(size=(n, 4)),
                scales2=np.exp(g.uniform(-3.0, -1.9, (n, 2))), opacities=g.uniform(0.1, 0.95, n),
                rgb=g.uniform(0, 1, (n, 3)))
    surf = {k: np.asarray(v, np.float32).astype(np.float64) for k, v in surf.items()}
    prm = dict(bg=(0.3, 0.2, 0.1))
    dC = g.normal(size=(44 * 52, 3))
    a = oracle.render_2dgs_bwd(surf, cam, prm, dC)
    b = oracle.render_2dgs_bwd_brute(surf, cam, prm, dC)
    for k in ("means", "quats", "scales2", "opacities", "rgb"):
        np.testing.assert_allclose(a[k], b[k], rtol=1e-10, atol=1e-12, err_msg=k)
    assert np.abs(b["means"]).max() > 1e-3


def test_surfel_pipeline_with_sh_colour_matches_central_differences():
    """Tiled surfel render with SH colour: the footprint backward plus the
    colour's view-direction term against central differences of the whole
    forward."""
    g = np.random.default_rng(17)
    cam = axis_camera(W=30, H=26, fx=28.0, t=(0.02, 0.01, 0.0))
    n, deg = 8, 1
    q = g.normal(size=(n, 4))
    sc = dict(means=g.normal(0, 0.25, (n, 3)) + [0, 0, 2.0], quats=q / np.linalg.norm(q, axis=1, keepdims=True),
              scales2=np.exp(g.uniform(-2.6, -1.7, (n, 2))), opacities=g.uniform(0.2, 0.9, n),
              sh=g.normal(0, 0.3, (n, 4, 3)), sh_degree=deg)
    sc["sh"][:, 0, :] += 1.0
    prm = dict(bg=(0.1, 0.2, 0.3))
    dC = g.normal(size=(26 * 30, 3))
    grads = oracle.surfel_backward(sc, cam, prm, dC)

    def loss(s):
        return float((oracle.surfel_forward(s, cam, prm)["rgb"].reshape(-1, 3) * dC).sum())

    checked = 0
    for key in ("means", "quats", "scales2", "opacities", "sh"):
        base = np.asarray(sc[key], np.float64)
        flat = base.reshape(-1)
        for i in range(flat.size):
            fds = []
            for h in (1e-6, 5e-7):
                vals = []
                for sgn in (1, -1):
                    pert = flat.copy()
                    pert[i] += sgn * h
                    vals.append(loss(dict(sc, **{key: pert.reshape(base.shape)})))
                fds.append((vals[0] - vals[1]) / (2 * h))
            if abs(fds[0] - fds[1]) > 1e-6 * max(1.0, abs(fds[0])):
                continue
            an = grads[key].reshape(-1)[i]
            assert abs(fds[0] - an) <= 2e-6 * max(1.0, abs(fds[0])), (key, i, fds[0], an)
            checked += abs(an) > 1e-8
    assert checked > 100


def test_ndfd_over_surfels():
    """NDFD on surfel weights: with a constant f_gt, L_gt is the surfel render
    of each surfel's sigma; the contributor counts are the render's; L_cf is
    the pair sum of Eq. 6 over each pixel's contributors, composited here
    directly from the ray-plane solve."""
    g = np.random.default_rng(18)
    cam = axis_camera(W=26, H=22, fx=24.0, t=(0.0, 0.01, 0.0))
    n, D = 30, 6
    surf = dict(means=g.normal(0, 0.3, (n, 3)) + [0, 0, 2.0], quats=g.normal(size=(n, 4)),
                scales2=np.exp(g.uniform(-2.6, -1.8, (n, 2))), opacities=g.uniform(0.2, 0.9, n))
    surf = {k: np.asarray(v, np.float32).astype(np.float64) for k, v in surf.items()}
    f = g.normal(size=(n, D))
    f /= np.linalg.norm(f, axis=1, keepdims=True)
    gt = g.normal(size=D)
    K, LAM = oracle.NDFD_K, oracle.NDFD_LAMBDA
    sig = 1.0 / (1.0 + np.exp(K * (f @ gt / np.linalg.norm(gt) - LAM)))
    out = oracle.ndfd_2dgs(surf, cam, {}, f, np.broadcast_to(gt, (22, 26, D)))
    ren = oracle.render_2dgs(dict(surf, rgb=np.stack([sig, 0 * sig, 0 * sig], 1)), cam, {})
    np.testing.assert_allclose(out["Lgt"], ren["rgb"][..., 0], atol=1e-13)
    np.testing.assert_array_equal(out["ncontrib"], ren["ncontrib"])
    # Eq. 6 pair sum with per-pixel ground truth
    fg = g.normal(size=(22, 26, D))
    out = oracle.ndfd_2dgs(surf, cam, {}, f, fg)
    lists = ren["lists"]
    ranges = lists["ranges"]
    checked = 0
    for y in range(22):
        for x in range(26):
            t = (y // 16) * 2 + x // 16
            ids = lists["gids"][ranges[t][0]:ranges[t][1]]
            uv = oracle.splat_uv(surf["means"][ids], surf["quats"][ids], surf["scales2"][ids], cam,
                                 np.full(len(ids), x + 0.5), np.full(len(ids), y + 0.5))
            T, ws, fs = 1.0, [], []
            for j, gid in enumerate(ids):
                if not uv["hit"][j] or uv["lam"][j] <= 0:
                    continue
                r2 = uv["u"][j] ** 2 + uv["v"][j] ** 2
                if r2 > 9:
                    continue
                a = min(0.99, surf["opacities"][gid] * math.exp(-0.5 * r2))
                if a < 1 / 255:
                    continue
                if T * (1 - a) < 1e-4:
                    break
                ws.append(a * T)
                fs.append(f[gid])
                T *= 1 - a
            s = [1.0 / (1.0 + math.exp(K * (fi @ fg[y, x] / np.linalg.norm(fg[y, x]) - LAM))) for fi in fs]
            lcf = sum(s[i] * ws[i] * ws[j] * (1 - fs[i] @ fs[j]) for i in range(len(ws)) for j in range(i))
            assert abs(out["Lcf"][y, x] - lcf) < 1e-13
            checked += len(ws) >= 3
    assert checked > 30


def test_ndfd_over_surfels_backward_matches_central_differences():
    g = np.random.default_rng(19)
    cam = axis_camera(W=24, H=22, fx=23.0, t=(0.01, 0.0, 0.0))
    n, D = 9, 5
    q = g.normal(size=(n, 4))
    surf = dict(means=g.normal(0, 0.25, (n, 3)) + [0, 0, 2.0], quats=q / np.linalg.norm(q, axis=1, keepdims=True),
                scales2=np.exp(g.uniform(-2.4, -1.7, (n, 2))), opacities=g.uniform(0.2, 0.9, n))
    f = g.normal(size=(n, D))
    f /= np.linalg.norm(f, axis=1, keepdims=True)
    fg = g.normal(size=(22, 24, D))
    a, b = g.normal(size=(22, 24)), g.normal(size=(22, 24))
    grads = oracle.ndfd_2dgs_bwd(surf, cam, {}, f, fg, a, b)

    def loss(s):
        r = oracle.ndfd_2dgs(s, cam, {}, f, fg)
        return float((r["Lgt"] * a).sum() + (r["Lcf"] * b).sum())

    checked = 0
    for key in ("means", "quats", "scales2", "opacities"):
        base = np.asarray(surf[key], np.float64)
        flat = base.reshape(-1)
        for i in range(flat.size):
            fds = []
            for h in (1e-6, 5e-7):
                vals = []
                for sgn in (1, -1):
                    pert = flat.copy()
                    pert[i] += sgn * h
                    vals.append(loss(dict(surf, **{key: pert.reshape(base.shape)})))
                fds.append((vals[0] - vals[1]) / (2 * h))
            if abs(fds[0] - fds[1]) > 1e-6 * max(1.0, abs(fds[0])):
                continue
            an = grads[key].reshape(-1)[i]
            assert abs(fds[0] - an) <= 2e-6 * max(1.0, abs(fds[0])), (key, i, fds[0], an)
            checked += abs(an) > 1e-8
    assert checked > 60


def test_surfel_binning_rule_covers_the_exact_box_at_1080p():
    """At the bench's scale (1920x1080, f = 1662.8, surfels at depth ~4 with
    log-scales U[-5, -2]) the binary32 rule's pixel rectangle contains the
    exact box's pixels for every binned surfel, with a few pixels of pad."""
    g = np.random.default_rng(1)
    cam = axis_camera(W=1920, H=1080, fx=1662.8, cx=960, cy=540)
    m = 50000
    mu = (g.normal(0, 0.6, (m, 3)) + [0, 0, 4.0]).astype(np.float32)
    q = g.normal(size=(m, 4)).astype(np.float32)
    s2 = np.exp(g.uniform(-5, -2, (m, 2))).astype(np.float32)
    b = oracle.bin_surfel_f32(mu, q, s2, cam)
    ex = oracle.surfel_rect(mu.astype(np.float64), q.astype(np.float64), s2.astype(np.float64), cam)
    ok = (b["ntiles"] > 0) & ex["bounded"]
    r, p = ex["rect"][ok], b["pix"][ok]
    xl, xh = np.maximum(np.ceil(r[:, 0] - 0.5), 0), np.minimum(np.floor(r[:, 1] - 0.5), 1919)
    yl, yh = np.maximum(np.ceil(r[:, 2] - 0.5), 0), np.minimum(np.floor(r[:, 3] - 0.5), 1079)
    valid = (xl <= xh) & (yl <= yh)
    assert valid.sum() > 40000
    assert not (valid & ((p[:, 0] > xl) | (p[:, 2] < xh) | (p[:, 1] > yl) | (p[:, 3] < yh))).any()
    over = np.maximum(np.maximum(xl - p[:, 0], p[:, 2] - xh), np.maximum(yl - p[:, 1], p[:, 3] - yh))[valid]
    assert np.median(over) <= 3


def _random_surfels(seed, n, W, H):
    g = np.random.default_rng(seed)
    surf = dict(means=g.normal(0, 0.35, (n, 3)) + [0, 0, 2.4], quats=g.normal(size=(n, 4)),
                scales2=np.exp(g.uniform(-3.0, -1.9, (n, 2))), opacities=g.uniform(0.1, 0.95, n),
                rgb=g.uniform(0, 1, (n, 3)))
    return {k: np.asarray(v, np.float32).astype(np.float64) for k, v in surf.items()}, g


def test_tiled_surfel_features_are_blended_with_the_weights():
    """Eq. 4's feature blend over surfels: a constant unit feature gives
    sum w = 1 - T at every pixel (the weights and the transmittance
    telescope), and the blend is linear in the features."""
    cam = axis_camera(W=48, H=40, fx=44.0, t=(0.01, -0.02, 0.0))
    surf, g = _random_surfels(21, 80, 48, 40)
    ones = np.ones((80, 1))
    out = oracle.render_2dgs(surf, cam, None, feats=ones)
    np.testing.assert_allclose(out["feat"][..., 0] + out["T"], 1.0, atol=1e-12)
    assert (out["ncontrib"] > 3).mean() > 0.2
    f1, f2 = g.normal(size=(80, 5)), g.normal(size=(80, 5))
    a = oracle.render_2dgs(surf, cam, None, feats=f1)["feat"]
    b = oracle.render_2dgs(surf, cam, None, feats=f2)["feat"]
    c = oracle.render_2dgs(surf, cam, None, feats=f1 + 2.0 * f2)["feat"]
    np.testing.assert_allclose(c, a + 2.0 * b, atol=1e-12)


def test_tiled_surfel_margin_covers_every_flipped_decision():
    """Moving alpha_min, the cutoff or t_eps by a relative 1e-3 changes the
    image only at pixels whose margin is below 1e-3."""
    cam = axis_camera(W=52, H=44, fx=46.0, t=(0.01, 0.02, 0.0))
    surf, _ = _random_surfels(22, 120, 52, 44)
    base = oracle.render_2dgs(surf, cam, None)
    changed_total = 0
    for key in ("alpha_min", "cutoff_sq", "t_eps"):
        for f in (1.0 - 1e-3, 1.0 + 1e-3):
            prm = {key: oracle.DEFAULT_PARAMS[key] * f}
            alt = oracle.render_2dgs(surf, cam, prm)
            changed = np.abs(alt["rgb"] - base["rgb"]).max(axis=-1) > 0
            assert np.all(base["margin"][changed] < 1e-3), key
            changed_total += int(changed.sum())
    assert changed_total > 0


def test_surfel_pipeline_with_features_matches_central_differences():
    """The surfel backward's feature term: dL/dw takes dF . f, and the
    feature gradient is sum_p w dF, against central differences of the
    whole forward (SH colour and features)."""
    g = np.random.default_rng(23)
    cam = axis_camera(W=26, H=22, fx=24.0, t=(0.02, 0.01, 0.0))
    n, D = 7, 3
    q = g.normal(size=(n, 4))
    sc = dict(means=g.normal(0, 0.25, (n, 3)) + [0, 0, 2.0], quats=q / np.linalg.norm(q, axis=1, keepdims=True),
              scales2=np.exp(g.uniform(-2.6, -1.7, (n, 2))), opacities=g.uniform(0.2, 0.9, n),
              sh=g.normal(0, 0.3, (n, 1, 3)), sh_degree=0)
    sc["sh"][:, 0, :] += 1.0
    feats = g.normal(size=(n, D))
    prm = dict(bg=(0.1, 0.2, 0.3))
    dC, dF = g.normal(size=(22 * 26, 3)), g.normal(size=(22 * 26, D))
    grads = oracle.surfel_backward(sc, cam, prm, dC, feats=feats, dF=dF)

    def loss(s, f):
        out = oracle.surfel_forward(s, cam, prm, feats=f)
        return float((out["rgb"].reshape(-1, 3) * dC).sum() + (out["feat"].reshape(-1, D) * dF).sum())

    checked = 0
    for key in ("means", "quats", "scales2", "opacities", "features"):
        base = np.asarray(feats if key == "features" else sc[key], np.float64)
        flat = base.reshape(-1)
        for i in range(flat.size):
            fds = []
            for h in (1e-6, 5e-7):
                vals = []
                for sgn in (1, -1):
                    pert = flat.copy()
                    pert[i] += sgn * h
                    pb = pert.reshape(base.shape)
                    vals.append(loss(sc, pb) if key == "features" else loss(dict(sc, **{key: pb}), feats))
                fds.append((vals[0] - vals[1]) / (2 * h))
            if abs(fds[0] - fds[1]) > 1e-6 * max(1.0, abs(fds[0])):
                continue
            an = grads[key].reshape(-1)[i]
            assert abs(fds[0] - an) <= 2e-6 * max(1.0, abs(fds[0])), (key, i, fds[0], an)
            checked += abs(an) > 1e-8
    assert checked > 40
