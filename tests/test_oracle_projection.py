"""Pins of the oracle's projection, SH colour and binning (no GPU).

Each test checks the oracle against something other than itself: closed
forms of the EWA footprint, scipy's spherical harmonics, quadrature
orthonormality, brute-force enumeration of covered pixels and tiles.
"""
import math

import numpy as np
import pytest
import scipy.special as sps

import oracle
from tests.helpers import axis_camera, scene_from, small_random_scene

P = dict(sh_degree=0)
DIL = 0.3


def test_isotropic_on_axis_closed_form():
    cam = axis_camera(W=64, H=48, fx=50.0, fy=60.0)
    s, z = 0.05, 3.0
    rec = oracle.project(scene_from([[0, 0, z]], s), cam, P)[0]
    va = (50.0 * s / z) ** 2 + DIL
    vc = (60.0 * s / z) ** 2 + DIL
    assert rec[oracle.R_VALID] == 1
    np.testing.assert_allclose([rec[oracle.R_A], rec[oracle.R_B], rec[oracle.R_C]],
                               [1 / va, 0.0, 1 / vc], rtol=1e-13, atol=1e-15)
    np.testing.assert_allclose([rec[oracle.R_MX], rec[oracle.R_MY]], [32.0, 24.0], rtol=0, atol=1e-12)
    assert rec[oracle.R_DEPTH] == z


def test_off_axis_jacobian_term():
    """A Gaussian at (tx, 0, tz): Sigma'_00 = s^2 fx^2 (1 + tx^2/tz^2)/tz^2 + dil."""
    cam = axis_camera(W=200, H=200, fx=100.0)
    s, tx, tz = 0.04, 0.6, 2.0
    rec = oracle.project(scene_from([[tx, 0, tz]], s), cam, P)[0]
    a = s * s * 100.0 ** 2 * (1 + tx * tx / tz ** 2) / tz ** 2 + DIL
    c = s * s * 100.0 ** 2 / tz ** 2 + DIL
    np.testing.assert_allclose([rec[oracle.R_SIG_A], rec[oracle.R_SIG_B], rec[oracle.R_SIG_C]],
                               [a, 0.0, c], rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(rec[oracle.R_MX], 100.0 * tx / tz + 100.0, rtol=1e-14)


def test_fov_clamp_of_jacobian():
    """Beyond 1.3 x tan(half FoV) the Jacobian uses the clamped ratio."""
    cam = axis_camera(W=100, H=100, fx=50.0)
    s, tz = 0.05, 2.0
    lim = 1.3 * (0.5 * 100 / 50.0)
    tx = 3.0 * tz  # ratio 3 > lim 1.3
    rec = oracle.project(scene_from([[tx, 0, tz]], s), cam, P)[0]
    a = s * s * 50.0 ** 2 * (1 + lim * lim) / tz ** 2 + DIL
    np.testing.assert_allclose(rec[oracle.R_SIG_A], a, rtol=1e-12)


def test_anisotropic_and_rotated():
    cam = axis_camera(W=64, H=64, fx=40.0)
    sx, sy, sz, z = 0.08, 0.02, 0.05, 2.5
    rec = oracle.project(scene_from([[0, 0, z]], [sx, sy, sz]), cam, P)[0]
    np.testing.assert_allclose([rec[oracle.R_SIG_A], rec[oracle.R_SIG_C]],
                               [(40 * sx / z) ** 2 + DIL, (40 * sy / z) ** 2 + DIL], rtol=1e-12)
    # 90 degrees about z swaps the x and y extents
    q = [math.cos(math.pi / 4), 0.0, 0.0, math.sin(math.pi / 4)]
    rec = oracle.project(scene_from([[0, 0, z]], [sx, sy, sz], quats=[q]), cam, P)[0]
    np.testing.assert_allclose([rec[oracle.R_SIG_A], rec[oracle.R_SIG_B], rec[oracle.R_SIG_C]],
                               [(40 * sy / z) ** 2 + DIL, 0.0, (40 * sx / z) ** 2 + DIL],
                               rtol=1e-12, atol=1e-12)
    # 45 degrees: off-diagonal = (sx^2 - sy^2)/2 (scaled), closed form
    q = [math.cos(math.pi / 8), 0.0, 0.0, math.sin(math.pi / 8)]
    rec = oracle.project(scene_from([[0, 0, z]], [sx, sy, sz], quats=[q]), cam, P)[0]
    k = (40 / z) ** 2
    np.testing.assert_allclose([rec[oracle.R_SIG_A], rec[oracle.R_SIG_B], rec[oracle.R_SIG_C]],
                               [k * (sx * sx + sy * sy) / 2 + DIL, k * (sx * sx - sy * sy) / 2,
                                k * (sx * sx + sy * sy) / 2 + DIL], rtol=1e-12)


def test_rotation_matrix_properties():
    g = np.random.default_rng(3)
    q = g.normal(size=(50, 4))
    R = oracle.quat_to_rot(q)
    for Ri in R:
        np.testing.assert_allclose(Ri @ Ri.T, np.eye(3), atol=1e-13)
        assert abs(np.linalg.det(Ri) - 1) < 1e-13
    np.testing.assert_allclose(oracle.quat_to_rot(-q), R, atol=1e-14)
    np.testing.assert_allclose(oracle.quat_to_rot(2.5 * q), R, atol=1e-14)
    # 90 degrees about z maps x to y
    R90 = oracle.quat_to_rot(np.array([[math.cos(math.pi / 4), 0, 0, math.sin(math.pi / 4)]]))[0]
    np.testing.assert_allclose(R90 @ [1, 0, 0], [0, 1, 0], atol=1e-15)


def test_quaternion_sign_and_scale_invariance():
    sc = small_random_scene(20, seed=1, sh_degree=1, D=0)
    cam = axis_camera(t=(0, 0, 3.0))
    r0 = oracle.project(sc, cam, dict(sh_degree=1))
    for f in (-1.0, 3.0):
        s2 = dict(sc)
        s2["quats"] = sc["quats"] * f
        np.testing.assert_allclose(oracle.project(s2, cam, dict(sh_degree=1)), r0, rtol=1e-12, atol=1e-13)


def test_mean2d_and_depth_closed_form_camera_pose():
    from paper_2505_19154_gb300 import synth
    cam = synth.look_at_camera([0.0, 0.0, -4.0], 64, 64)
    X = np.array([[0.3, -0.2, 0.5]])
    rec = oracle.project(scene_from(X, 0.01), cam, P)[0]
    fx = 32.0 / math.tan(math.radians(30))
    np.testing.assert_allclose([rec[oracle.R_MX], rec[oracle.R_MY], rec[oracle.R_DEPTH]],
                               [fx * 0.3 / 4.5 + 32, fx * -0.2 / 4.5 + 32, 4.5], rtol=1e-12)


def test_near_plane_cull():
    cam = axis_camera()
    rec = oracle.project(scene_from([[0, 0, 0.1], [0, 0, 0.2], [0, 0, 0.21]], 0.01), cam, P)
    assert list(rec[:, oracle.R_VALID]) == [0, 0, 1]


# -------------------------------------------------------------------- SH
def _real_sh_scipy(l, m, dirs):
    x, y, z = dirs.T
    theta = np.arccos(np.clip(z, -1, 1))
    phi = np.arctan2(y, x)
    if m == 0:
        return sps.sph_harm_y(l, 0, theta, phi).real
    Y = sps.sph_harm_y(l, abs(m), theta, phi)
    return math.sqrt(2.0) * (Y.real if m > 0 else Y.imag)


def test_sh_basis_matches_scipy_up_to_sign():
    g = np.random.default_rng(0)
    d = g.normal(size=(200, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    Y, _ = oracle.sh_basis(d)
    idx = 0
    for l in range(4):
        for m in range(-l, l + 1):
            ref = _real_sh_scipy(l, m, d)
            sign = np.sign(np.dot(ref, Y[:, idx]))
            assert sign != 0
            np.testing.assert_allclose(Y[:, idx], sign * ref, atol=1e-12, err_msg=f"l={l} m={m}")
            idx += 1


def test_sh_orthonormal_by_quadrature():
    # Gauss-Legendre in cos(theta) x uniform phi: exact for these polynomials
    xg, wg = np.polynomial.legendre.leggauss(12)
    nphi = 24
    phi = (np.arange(nphi) + 0.5) * 2 * np.pi / nphi
    ct, ph = np.meshgrid(xg, phi, indexing="ij")
    st = np.sqrt(1 - ct ** 2)
    d = np.stack([st * np.cos(ph), st * np.sin(ph), ct], -1).reshape(-1, 3)
    w = (wg[:, None] * np.full(nphi, 2 * np.pi / nphi)[None, :]).reshape(-1)
    Y, _ = oracle.sh_basis(d)
    G = (Y * w[:, None]).T @ Y
    np.testing.assert_allclose(G, np.eye(16), atol=1e-12)


def test_sh_gradient_by_finite_differences():
    g = np.random.default_rng(1)
    d = g.normal(size=(30, 3))
    _, dY = oracle.sh_basis(d)
    h = 1e-6
    for k in range(3):
        e = np.zeros(3)
        e[k] = h
        fd = (oracle.sh_basis(d + e)[0] - oracle.sh_basis(d - e)[0]) / (2 * h)
        np.testing.assert_allclose(dY[:, :, k], fd, atol=1e-7)


def test_sh_colour_degree0_and_clamp():
    cam = axis_camera()
    colors = np.array([[0.2, 0.7, 1.3], [-0.4, 0.5, 0.0]])
    sc = scene_from([[0, 0, 2.0], [0.1, 0, 2.0]], 0.05, colors=colors)
    rec = oracle.project(sc, cam, P)
    np.testing.assert_allclose(rec[:, oracle.R_RAW_R:oracle.R_RAW_B + 1], colors, atol=1e-14)
    np.testing.assert_allclose(rec[:, oracle.R_R:oracle.R_BL + 1], np.maximum(colors, 0), atol=1e-14)


def test_sh_view_direction_degree1():
    """Degree 1 at the +z axis direction: only Y_{1,0} = C1 z is non-zero."""
    cam = axis_camera()
    sh = np.zeros((1, 4, 3))
    sh[0, 2] = [1.0, -1.0, 0.5]   # coefficient of C1*z
    sc = scene_from([[0, 0, 2.0]], 0.05, sh=sh)
    rec = oracle.project(sc, cam, dict(sh_degree=1))[0]
    c1 = math.sqrt(3 / (4 * math.pi))
    np.testing.assert_allclose(rec[oracle.R_RAW_R:oracle.R_RAW_B + 1], 0.5 + c1 * np.array([1.0, -1.0, 0.5]),
                               atol=1e-14)


# --------------------------------------------------------------- binning
def _brute_rect_check(sc, cam, prm):
    """Every pixel whose centre is inside the FP64 ellipse (q2 <= 9, margin
    excluded) must be inside the FP32 pixel rectangle; and the rectangle
    must be tight (each edge row/column meets the ellipse up to rounding)."""
    b = oracle.bin_f32(sc, cam, prm)
    rec = oracle.project(sc, cam, prm)
    W, H = cam["width"], cam["height"]
    ys, xs = np.mgrid[0:H, 0:W]
    bad = 0
    for g in range(len(rec)):
        r = rec[g]
        if r[oracle.R_VALID] == 0:
            assert b["ntiles"][g] == 0
            continue
        dx = xs + 0.5 - r[oracle.R_MX]
        dy = ys + 0.5 - r[oracle.R_MY]
        q2 = r[oracle.R_A] * dx * dx + 2 * r[oracle.R_B] * dx * dy + r[oracle.R_C] * dy * dy
        inside = q2 <= 9.0 * (1 - 1e-6)
        if not inside.any():
            continue
        x0, y0, x1, y1 = b["pix"][g]
        covered = (xs >= x0) & (xs <= x1) & (ys >= y0) & (ys <= y1)
        bad += int((inside & ~covered).sum())
        # tight: the ellipse's exact bounding box, rounded to pixel centres
        ex, ey = r[oracle.R_EXT_X], r[oracle.R_EXT_Y]
        assert x0 == max(0, math.ceil(r[oracle.R_MX] - ex - 0.5)) or abs((r[oracle.R_MX] - ex - 0.5) % 1) < 1e-4
        assert y1 == min(H - 1, math.floor(r[oracle.R_MY] + ey - 0.5)) or abs((r[oracle.R_MY] + ey - 0.5) % 1) < 1e-4
        tx0, ty0, tx1, ty1 = b["tile"][g]
        assert (tx0, ty0, tx1, ty1) == (x0 // 16, y0 // 16, x1 // 16, y1 // 16)
        assert b["ntiles"][g] == (tx1 - tx0 + 1) * (ty1 - ty0 + 1)
        # FP32 depth: a few binary32 roundings away from the FP64 depth
        assert abs(int(b["dbits"][g]) - int(np.float32(r[oracle.R_DEPTH]).view(np.uint32))) <= 4
    assert bad == 0


def test_bin_rect_covers_fp64_ellipse():
    sc = small_random_scene(60, seed=2, sh_degree=0, D=0, spread=0.6)
    cam = axis_camera(W=80, H=56, fx=60.0, t=(0.05, -0.03, 2.5))
    _brute_rect_check(sc, cam, P)


def test_bin_fp32_footprint_close_to_fp64():
    from paper_2505_19154_gb300 import synth
    sc, cams = synth.config2(0)
    sub = {k: (v[:5000] if isinstance(v, np.ndarray) else v) for k, v in sc.items()}
    b = oracle.bin_f32(sub, cams[0], dict(sh_degree=3))
    rec = oracle.project(sub, cams[0], dict(sh_degree=3))
    ok = (b["ntiles"] > 0)
    v64 = rec[:, oracle.R_VALID] > 0
    assert (ok <= v64).all()
    np.testing.assert_allclose(b["fp"][ok][:, 0], rec[ok, oracle.R_MX], rtol=2e-6, atol=2e-4)
    np.testing.assert_allclose(b["fp"][ok][:, 2], rec[ok, oracle.R_A], rtol=1e-4)


def test_tile_lists_match_brute_force_membership_and_order():
    sc = small_random_scene(80, seed=4, sh_degree=0, D=0, spread=0.7)
    cams = [axis_camera(W=70, H=50, fx=50.0, t=(0, 0, 2.5)), axis_camera(W=33, H=47, fx=30.0, t=(0.2, 0, 2.0))]
    bins = [oracle.bin_f32(sc, c, P) for c in cams]
    L = oracle.tile_lists(bins, cams, P)
    keys, gids, ranges = L["keys"], L["gids"], L["ranges"]
    # sorted by (key, gid)
    order = sorted(range(len(keys)), key=lambda i: (int(keys[i]), int(gids[i])))
    assert order == list(range(len(keys)))
    offs = L["cam_tile_offset"]
    for ci, (cam, b) in enumerate(zip(cams, bins)):
        tx_n, ty_n = oracle.tiles_xy(cam)
        for ty in range(ty_n):
            for tx in range(tx_n):
                t = offs[ci] + ty * tx_n + tx
                s, e = ranges[t]
                got = list(gids[s:e])
                want = [g for g in range(len(sc["means"])) if b["ntiles"][g] > 0
                        and b["tile"][g][0] <= tx <= b["tile"][g][2] and b["tile"][g][1] <= ty <= b["tile"][g][3]]
                want.sort(key=lambda g: (int(b["dbits"][g]), g))
                assert got == want
                for i in range(s, e):
                    assert int(keys[i]) == (t << 32) | int(b["dbits"][gids[i]])


def test_tile_rect_window_is_a_restriction():
    sc = small_random_scene(60, seed=5, sh_degree=0, D=0, spread=0.6)
    cam = axis_camera(W=96, H=64, fx=60.0, t=(0, 0, 2.5))
    b = [oracle.bin_f32(sc, cam, P)]
    full = oracle.tile_lists(b, [cam], P)
    win = oracle.tile_lists(b, [cam], P, tile_rect=(1, 1, 3, 2))
    for ty in range(1, 3):
        for tx in range(1, 4):
            t = ty * 6 + tx
            s, e = full["ranges"][t]
            s2, e2 = win["ranges"][t]
            assert list(full["gids"][s:e]) == list(win["gids"][s2:e2])
