"""Pins of the oracle's compositing (Eq. 4), its derivative and fusion (no GPU).

(a) a lone Gaussian's peak equals opacity x colour (+ background through the
    remaining transmittance), and its profile is the closed-form Gaussian;
(b) the compositing weights plus the final transmittance sum to 1;
(c) per-pixel brute-force depth-sorted compositing (no tiles) equals the
    tiled result;
(d) fusing a constant feature map returns that constant;
plus hand-computed compositing fixtures, the transmittance stop rule,
finite differences of the whole forward, and the App. A.2 identity.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle
from paper_2505_19154_gb300 import synth
from tests.helpers import axis_camera, scene_from, small_random_scene

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _render_all(sc, cam, prm, feats=None):
    prep = oracle.prepare(sc, [cam], prm)
    return oracle.forward(sc, [cam], prm, feats, prep=prep)[0], prep


def test_lone_gaussian_peak_and_profile():
    # mean lands exactly on the centre of pixel (32, 20): cx = 32.5, cy = 20.5
    cam = axis_camera(W=64, H=40, fx=80.0, cx=32.5, cy=20.5)
    s, z, op = 0.06, 2.0, 0.7
    col = np.array([0.9, 0.3, 0.6])
    f = np.array([[1.5, -2.0, 0.25]])
    prm = dict(sh_degree=0, bg=(0.1, 0.2, 0.3))
    sc = scene_from([[0, 0, z]], s, opac=op, colors=[col], feats=f)
    out, _ = _render_all(sc, cam, prm, f)
    peak = out["rgb"][20, 32]
    np.testing.assert_allclose(peak, op * col + (1 - op) * np.array([0.1, 0.2, 0.3]), rtol=0, atol=1e-14)
    np.testing.assert_allclose(out["feat"][20, 32], op * f[0], atol=1e-14)
    # profile: alpha(d) = op exp(-d^2 / (2 (sigma_px^2 + 0.3)))
    var = (80.0 * s / z) ** 2 + 0.3
    for (py, px) in [(20, 33), (21, 32), (22, 34), (17, 30)]:
        d2 = (px - 32) ** 2 + (py - 20) ** 2
        a = op * math.exp(-d2 / (2 * var))
        if a < 1 / 255 or d2 / var > 9:
            a = 0.0
        np.testing.assert_allclose(out["feat"][py, px], a * f[0], atol=1e-14)
        np.testing.assert_allclose(out["T"][py, px], 1 - a, atol=1e-14)


def test_weights_plus_transmittance_is_one():
    sc = small_random_scene(120, seed=7, sh_degree=2, D=0, spread=0.4)
    cam = axis_camera(W=48, H=40, fx=40.0, t=(0, 0, 2.2))
    ones = np.ones((120, 1))
    out, _ = _render_all(sc, cam, dict(sh_degree=2), ones)
    np.testing.assert_allclose(out["feat"][..., 0] + out["T"], 1.0, atol=1e-12)
    assert (out["ncontrib"] > 3).mean() > 0.3   # the scene really overlaps


def test_bruteforce_equals_tiled():
    sc = small_random_scene(150, seed=8, sh_degree=3, D=5, spread=0.45)
    cam = axis_camera(W=72, H=56, fx=45.0, t=(0.05, -0.02, 2.4))
    prm = dict(sh_degree=3, bg=(0.2, 0.1, 0.0))
    out, prep = _render_all(sc, cam, prm, sc["features"])
    rec = prep["recs"][0]
    dk = prep["bins"][0]["dbits"].astype(np.float64)   # same order key as the tiles
    br = oracle.render_brute(rec, dk, sc["features"], cam, prm)
    ok = (out["margin"] > 1e-5) & (br["margin"] > 1e-5)
    assert ok.mean() > 0.99
    np.testing.assert_allclose(out["rgb"][ok], br["rgb"][ok], atol=1e-12)
    np.testing.assert_allclose(out["feat"][ok], br["feat"][ok], atol=1e-12)
    np.testing.assert_allclose(out["T"][ok], br["T"][ok], atol=1e-12)


def test_feature_linearity_and_unit_features_give_weights():
    sc = small_random_scene(60, seed=9, sh_degree=0, D=0, spread=0.4)
    cam = axis_camera(W=40, H=40, fx=35.0, t=(0, 0, 2.2))
    g = np.random.default_rng(0)
    f1, f2 = g.normal(size=(60, 3)), g.normal(size=(60, 3))
    prm = dict(sh_degree=0)
    a, prep = _render_all(sc, cam, prm, f1)
    b = oracle.forward(sc, [cam], prm, f2, prep=prep)[0]
    c = oracle.forward(sc, [cam], prm, f1 + f2, prep=prep)[0]
    np.testing.assert_allclose(c["feat"], a["feat"] + b["feat"], atol=1e-12)
    # f = e_k recovers the weight of Gaussian k
    k = int(np.argmax(sc["opacities"]))
    e = np.zeros((60, 1))
    e[k, 0] = 1.0
    wk = oracle.forward(sc, [cam], prm, e, prep=prep)[0]["feat"][..., 0]
    assert wk.max() > 0.05


def test_golden_compositing_fixture():
    """Hand-computed front-to-back compositing of three stacked Gaussians."""
    fx = json.load(open(os.path.join(GOLDEN, "compositing_three_stacked.json")))
    cam = axis_camera(W=8, H=8, fx=10.0, cx=4.5, cy=4.5)
    means = [[0, 0, z] for z in fx["depths"]]
    sc = scene_from(means, 0.01, opac=fx["opacities"], colors=fx["colors"], feats=fx["features"])
    prm = dict(sh_degree=0, bg=tuple(fx["background"]))
    out, _ = _render_all(sc, cam, prm, np.array(fx["features"]))
    np.testing.assert_allclose(out["rgb"][4, 4], fx["expected_rgb"], atol=1e-12)
    np.testing.assert_allclose(out["feat"][4, 4], fx["expected_feat"], atol=1e-12)
    np.testing.assert_allclose(out["T"][4, 4], fx["expected_T"], atol=1e-12)


def test_equal_depth_tie_is_ascending_index():
    cam = axis_camera(W=8, H=8, fx=10.0, cx=4.5, cy=4.5)
    sc = scene_from([[0, 0, 2.0], [0, 0, 2.0]], 0.01, opac=[0.6, 0.6],
                    colors=[[1, 0, 0], [0, 0, 1]])
    out, _ = _render_all(sc, cam, dict(sh_degree=0))
    np.testing.assert_allclose(out["rgb"][4, 4], [0.6, 0.0, 0.6 * 0.4], atol=1e-14)


def test_transmittance_stop_rule():
    """alpha = 0.95 stacked: T = 1, .05, .0025, .000125, then T' < 1e-4 stops."""
    cam = axis_camera(W=8, H=8, fx=10.0, cx=4.5, cy=4.5)
    n = 6
    sc = scene_from([[0, 0, 2.0 + 0.1 * i] for i in range(n)], 0.01, opac=0.95,
                    colors=[[1.0, 1.0, 1.0]] * n)
    out, _ = _render_all(sc, cam, dict(sh_degree=0))
    assert out["ncontrib"][4, 4] == 3 and out["last"][4, 4] == 3
    np.testing.assert_allclose(out["T"][4, 4], 0.05 ** 3, rtol=1e-12)
    np.testing.assert_allclose(out["rgb"][4, 4], 1 - 0.05 ** 3, rtol=1e-12)
    # traversal ends at the first failing test: a faint Gaussian behind the
    # stopping one (T' = 1.25e-4 * 0.9 >= 1e-4 on its own) is not composited
    op = [0.95, 0.95, 0.95, 0.95, 0.1]
    sc = scene_from([[0, 0, 2.0 + 0.1 * i] for i in range(5)], 0.01, opac=op,
                    colors=[[1.0, 1.0, 1.0]] * 5)
    out, _ = _render_all(sc, cam, dict(sh_degree=0))
    assert out["ncontrib"][4, 4] == 3 and out["last"][4, 4] == 3
    np.testing.assert_allclose(out["T"][4, 4], 0.05 ** 3, rtol=1e-12)


def test_alpha_threshold_and_ellipse_cutoff():
    cam = axis_camera(W=16, H=16, fx=10.0, cx=8.5, cy=8.5)
    # opacity 0.003 < 1/255: never contributes
    sc = scene_from([[0, 0, 2.0]], 0.2, opac=0.003)
    out, _ = _render_all(sc, cam, dict(sh_degree=0))
    assert (out["ncontrib"] == 0).all()
    # op 0.99: alpha at q2 = 9 is 0.99 e^-4.5 > 1/255, yet the cutoff removes
    # every pixel beyond the 3-sigma ellipse
    s, z = 0.2, 2.0
    var = (10 * s / z) ** 2 + 0.3
    sc = scene_from([[0, 0, z]], s, opac=0.99)
    out, _ = _render_all(sc, cam, dict(sh_degree=0))
    ys, xs = np.mgrid[0:16, 0:16]
    q2 = ((xs - 8) ** 2 + (ys - 8) ** 2) / var
    assert ((out["ncontrib"] > 0) == (q2 <= 9)).all()


# ---------------------------------------------------------------- backward
def _loss_brute(sc, cam, prm, feats, dC, dF, dkey):
    rec = oracle.project(sc, cam, prm)
    br = oracle.render_brute(rec, dkey, feats, cam, prm)
    L = float((br["rgb"].reshape(-1, 3) * dC).sum())
    if feats is not None:
        L += float((br["feat"].reshape(-1, feats.shape[1]) * dF).sum())
    return L, br["sig"]


@pytest.mark.parametrize("seed,opaque", [(11, False), (12, False), (13, True)])
def test_backward_matches_central_differences(seed, opaque):
    sc = small_random_scene(14, seed=seed, sh_degree=3, D=4, spread=0.35)
    sc["opacities"] = np.clip(sc["opacities"], 0.05, 0.9)
    if opaque:
        # near-opaque Gaussians: alpha = min(0.99, op G) clamps near centres
        sc["opacities"][::2] = np.linspace(0.991, 0.999, 7)
    cam = axis_camera(W=32, H=32, fx=30.0, t=(0.03, 0.02, 2.0))
    prm = dict(sh_degree=3, bg=(0.3, 0.1, 0.2))
    g = np.random.default_rng(seed)
    npx = 32 * 32
    dC, dF = g.normal(size=(npx, 3)), g.normal(size=(npx, 4))
    feats = sc["features"]
    grads = oracle.backward(sc, [cam], prm, feats, [dC], [dF])
    dkey = oracle.bin_f32(sc, cam, prm)["dbits"].astype(np.float64)
    _, sig0 = _loss_brute(sc, cam, prm, feats, dC, dF, dkey)
    checked = 0
    for name, key in [("means", "means"), ("scales", "scales"), ("quats", "quats"),
                      ("opacities", "opacities"), ("sh", "sh"), ("features", "features")]:
        base = np.asarray(sc[key], np.float64)
        flat = base.reshape(-1)
        for i in range(flat.size):
            h = 1e-6 * max(1.0, abs(flat[i]))
            vals = []
            same = True
            for sgn in (1, -1):
                pert = flat.copy()
                pert[i] += sgn * h
                s2 = dict(sc)
                s2[key] = pert.reshape(base.shape)
                f2 = s2["features"]
                L, sig = _loss_brute(s2, cam, prm, f2, dC, dF, dkey)
                same &= bool((sig == sig0).all())
                vals.append(L)
            if not same:
                continue
            fd = (vals[0] - vals[1]) / (2 * h)
            an = grads[name].reshape(-1)[i]
            assert abs(fd - an) <= 1e-5 * max(1.0, abs(fd)), (name, i, fd, an)
            checked += 1
    assert checked > 500


def test_dw_dalpha_identity_appendix():
    """dL/dalpha_k = T_k g_k - (1/(1-alpha_k)) sum_{i>k} w_i g_i (App. A.2),
    checked against central differences of w(alpha) = alpha_i prod_{j<i}(1-alpha_j)."""
    g = np.random.default_rng(5)
    a = g.uniform(0.05, 0.9, 9)
    gw = g.normal(size=9)

    def L(al):
        T = np.concatenate([[1.0], np.cumprod(1 - al)[:-1]])
        return float((al * T * gw).sum())

    T = np.concatenate([[1.0], np.cumprod(1 - a)[:-1]])
    w = a * T
    for k in range(9):
        e = np.zeros(9)
        e[k] = 1e-7
        fd = (L(a + e) - L(a - e)) / 2e-7
        formula = T[k] * gw[k] - (w[k + 1:] * gw[k + 1:]).sum() / (1 - a[k])
        assert abs(fd - formula) < 1e-7


def test_quat_gradient_orthogonal_to_quat():
    sc = small_random_scene(30, seed=13, sh_degree=1, D=2, spread=0.4)
    cam = axis_camera(W=40, H=40, fx=35.0, t=(0, 0, 2.2))
    g = np.random.default_rng(1)
    dC, dF = g.normal(size=(1600, 3)), g.normal(size=(1600, 2))
    gr = oracle.backward(sc, [cam], dict(sh_degree=1), sc["features"], [dC], [dF])
    dots = (gr["quats"] * sc["quats"]).sum(1)
    assert np.abs(dots).max() < 1e-12 * max(1.0, np.abs(gr["quats"]).max())


def test_backward_is_linear_in_upstream_and_sums_over_cameras():
    sc = small_random_scene(30, seed=14, sh_degree=1, D=2, spread=0.4)
    cams = [axis_camera(W=24, H=24, fx=20.0, t=(0, 0, 2.2)), axis_camera(W=20, H=28, fx=22.0, t=(0.1, 0, 2.0))]
    prm = dict(sh_degree=1)
    g = np.random.default_rng(2)
    dC = [g.normal(size=(24 * 24, 3)), g.normal(size=(20 * 28, 3))]
    dF = [g.normal(size=(24 * 24, 2)), g.normal(size=(20 * 28, 2))]
    both = oracle.backward(sc, cams, prm, sc["features"], dC, dF)
    one = oracle.backward(sc, cams[:1], prm, sc["features"], dC[:1], dF[:1])
    two = oracle.backward(sc, cams[1:], prm, sc["features"], dC[1:], dF[1:])
    for k in ("means", "scales", "quats", "opacities", "sh", "features"):
        np.testing.assert_allclose(both[k], one[k] + two[k], atol=1e-12)


# ------------------------------------------------------------------ fusion
def test_fuse_constant_map_returns_constant():
    sc = small_random_scene(80, seed=15, sh_degree=0, D=0, spread=0.4)
    views = [axis_camera(W=40, H=32, fx=30.0, t=(0, 0, 2.3)), axis_camera(W=36, H=36, fx=30.0, t=(-0.1, 0.05, 2.0))]
    c = np.array([0.3, -1.25, 2.0, 0.5])
    maps = [np.broadcast_to(c, (v["height"], v["width"], 4)) for v in views]
    out = oracle.fuse(sc, views, maps, dict(sh_degree=0))
    seen = out["den"] > 1e-9
    assert seen.sum() > 20
    np.testing.assert_allclose(out["out"][seen], np.broadcast_to(c, (seen.sum(), 4)), rtol=1e-13)
    assert (out["flag"][~seen] == 1).all() and (out["out"][~seen] == 0).all()


def test_fuse_single_gaussian_weighted_mean_and_shard_additivity():
    cam = axis_camera(W=20, H=20, fx=40.0, cx=10.5, cy=10.5)
    sc = scene_from([[0, 0, 2.0]], 0.1, opac=0.8)
    H = W = 20
    ys, xs = np.mgrid[0:H, 0:W]
    fmap = np.stack([xs + 0.5, ys + 0.5, np.ones_like(xs)], -1).astype(np.float64)
    out = oracle.fuse(sc, [cam], [fmap], dict(sh_degree=0))
    # symmetric footprint about the pixel centre (10.5, 10.5): the weighted
    # mean of x and y is the centre itself, and of the constant channel 1
    np.testing.assert_allclose(out["out"][0], [10.5, 10.5, 1.0], atol=1e-12)
    # additivity over view shards
    sc2 = small_random_scene(50, seed=16, sh_degree=0, D=0, spread=0.4)
    views = [axis_camera(W=24, H=24, fx=20.0, t=(0, 0, 2.2)), axis_camera(W=24, H=20, fx=25.0, t=(0.1, 0, 2.0))]
    g = np.random.default_rng(3)
    maps = [g.normal(size=(v["height"], v["width"], 3)) for v in views]
    a = oracle.fuse(sc2, views[:1], maps[:1], dict(sh_degree=0))
    b = oracle.fuse(sc2, views[1:], maps[1:], dict(sh_degree=0))
    ab = oracle.fuse(sc2, views, maps, dict(sh_degree=0))
    np.testing.assert_allclose(ab["num"], a["num"] + b["num"], atol=1e-12)
    np.testing.assert_allclose(ab["den"], a["den"] + b["den"], atol=1e-12)


def test_rotated_anisotropic_profile_closed_form():
    """45-degree rotated anisotropic Gaussian: alpha(d) = op exp(-d^T S^-1 d / 2)
    with S = k R diag(sx^2, sy^2) R^T + 0.3 I in closed form (k = (fx/z)^2)."""
    cam = axis_camera(W=64, H=64, fx=40.0, cx=32.5, cy=32.5)
    sx, sy, z, op = 0.3, 0.08, 2.0, 0.9
    q = [math.cos(math.pi / 8), 0.0, 0.0, math.sin(math.pi / 8)]
    sc = scene_from([[0, 0, z]], [sx, sy, 0.05], quats=[q], opac=op)
    out, _ = _render_all(sc, cam, dict(sh_degree=0), np.ones((1, 1)))
    k = (40.0 / z) ** 2
    S = np.array([[k * (sx * sx + sy * sy) / 2 + 0.3, k * (sx * sx - sy * sy) / 2],
                  [k * (sx * sx - sy * sy) / 2, k * (sx * sx + sy * sy) / 2 + 0.3]])
    Si = np.linalg.inv(S)
    for (dx, dy) in [(3, 3), (3, -3), (-5, -4), (0, 6), (7, 1)]:
        d = np.array([dx, dy], float)
        q2 = d @ Si @ d
        a = op * math.exp(-0.5 * q2)
        if a < 1 / 255 or q2 > 9:
            a = 0.0
        np.testing.assert_allclose(out["feat"][32 + dy, 32 + dx, 0], a, atol=1e-13, err_msg=str((dx, dy)))
    # the two diagonals really differ (the off-diagonal term matters)
    assert abs(out["feat"][35, 35, 0] - out["feat"][29, 35, 0]) > 0.05


def test_fusion_flip_bound_covers_threshold_perturbations():
    """The fusion margin diagnostic (wflip) bounds the weight any flipped
    near-threshold decision moves: moving alpha_min, the q^2 cutoff or t_eps
    by 0.5 % flips exactly the decisions within 0.5 % of their threshold, and
    every Gaussian's change of sum w (and of sum w F, unit-norm F) stays
    within its wflip computed with a 1 % tolerance; the fused feature then
    moves by at most 2 wflip / (den - wflip)."""
    sc = small_random_scene(500, seed=61, sh_degree=0, D=0, spread=0.45)
    views = [synth.look_at_camera(synth.ring_position(2.2, a, e), 48, 40) for a, e in [(10, 5), (150, -20)]]
    g = np.random.default_rng(9)
    maps = []
    for v in views:
        m = g.normal(size=(v["height"], v["width"], 4))
        maps.append(m / np.linalg.norm(m, axis=-1, keepdims=True))
    base = dict(sh_degree=0)
    prep = oracle.prepare(sc, views, base)
    ref = oracle.fuse(sc, views, maps, base, prep=prep, margin_tol=1e-2)
    assert (ref["den"] > 0).sum() > 100
    moved = 0
    for key in ("alpha_min", "cutoff_sq", "t_eps"):
        for f in (1.0 - 5e-3, 1.0 + 5e-3):
            prm = dict(base, **{key: oracle.DEFAULT_PARAMS[key] * f})
            alt = oracle.fuse(sc, views, maps, prm, prep=prep, margin_tol=0.0)
            d_den = np.abs(alt["den"] - ref["den"])
            d_num = np.linalg.norm(alt["num"] - ref["num"], axis=1)
            assert np.all(d_den <= ref["wflip"] * (1 + 1e-9) + 1e-15), (key, f)
            assert np.all(d_num <= ref["wflip"] * (1 + 1e-9) + 1e-15), (key, f)
            # the fused feature num/den moves by at most 2 wflip / (den - wflip)
            # (|F| = 1 >= |out|): the allowance the GPU fusion tests grant
            both = (ref["den"] > 1e-6) & (alt["den"] > 1e-6) & (ref["wflip"] < 0.5 * ref["den"])
            d_out = np.linalg.norm(alt["out"] - ref["out"], axis=1)
            allow = 2.0 * ref["wflip"] / np.maximum(ref["den"] - ref["wflip"], 1e-30)
            assert np.all(d_out[both] <= allow[both] * (1 + 1e-9) + 1e-15), (key, f)
            moved += int((d_den > 1e-12).sum())
    assert moved > 10  # the perturbations do flip decisions
    assert np.all(oracle.fuse(sc, views, maps, base, prep=prep, margin_tol=0.0)["wflip"] == 0.0)


def test_fp32_geometry_option_changes_only_the_footprint():
    """prepare(geometry="fp32") composites over the FP32 specification's mean
    and conic: same lists, records equal to the specification's values,
    images within FP32 rounding of the FP64-geometry render."""
    sc = small_random_scene(300, seed=71, sh_degree=1, D=3, spread=0.5)
    cam = synth.look_at_camera(synth.ring_position(2.5, 30, 10), 40, 32)
    prm = dict(sh_degree=1)
    p64 = oracle.prepare(sc, [cam], prm)
    p32 = oracle.prepare(sc, [cam], prm, geometry="fp32")
    np.testing.assert_array_equal(p64["lists"]["gids"], p32["lists"]["gids"])
    ok = p32["bins"][0]["ntiles"] > 0
    np.testing.assert_array_equal(p32["recs"][0][ok][:, :5], p32["bins"][0]["fp"][ok][:, :5].astype(np.float64))
    r32, r64 = p32["recs"][0][ok], p64["recs"][0][ok]
    assert np.abs(r32[:, :2] - r64[:, :2]).max() < 1e-3  # mean, pixels
    scale = np.maximum(np.abs(r64[:, 2]), np.abs(r64[:, 4]))[:, None]
    assert (np.abs(r32[:, 2:5] - r64[:, 2:5]) / scale).max() < 1e-4  # conic, relative to its size
    a = oracle.forward(sc, [cam], prm, sc["features"], prep=p64)[0]
    b = oracle.forward(sc, [cam], prm, sc["features"], prep=p32)[0]
    ok_px = (a["margin"] > 1e-4) & (b["margin"] > 1e-4)
    assert np.abs(a["rgb"] - b["rgb"])[ok_px].max() < 1e-4
    with pytest.raises(ValueError):
        oracle.prepare(sc, [cam], prm, geometry="fp16")
