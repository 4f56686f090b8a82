"""Pins of the oracle's NDFD losses and their derivative (no GPU).

L_gt = sum_i w_i sigma_i (Eq. 5) and L_cf = sum_i sigma_i w_i (W_{i-1} -
F_{i-1} . f_i) (Eq. 6), sigma_i = 1 / (1 + exp(k (cos<f_i, f_gt> - lambda)))
with k = 20, lambda = 0.5 (Sec. 3.3, Sec. 4), over the render's weights with
index 1 the nearest primitive.  Pinned by:
(a) the activation's closed values (sigma(lambda) = 1/2, the two ends);
(b) a two-Gaussian closed form that also fixes the order (nearest first);
(c) L_gt equal to the Eq. 4 render of the per-Gaussian sigma when f_gt is
    constant over the image;
(d) the O(N) recursion equal to the O(N^2) pair sum of Eq. 6's first line,
    brute force over each pixel's contributors;
(e) identical features give L_cf = 0; mutually orthogonal features with a
    common sigma give sigma ((sum w)^2 - sum w^2) / 2;
(f) the backward against central differences of the whole forward, and for
    L_gt alone against the (already pinned) render backward of sigma.
"""
import math

import numpy as np
import pytest

import oracle
from tests.helpers import axis_camera, scene_from, small_random_scene

K, LAM = oracle.NDFD_K, oracle.NDFD_LAMBDA


def _unit(a):
    a = np.asarray(a, np.float64)
    return a / np.linalg.norm(a, axis=-1, keepdims=True)


def _run(sc, cam, prm, fgt):
    prep = oracle.prepare(sc, [cam], prm)
    out = oracle.ndfd_forward(sc, [cam], prm, sc["features"], [fgt], prep=prep)[0]
    return out, prep


def test_activation_closed_values_on_a_lone_gaussian():
    cam = axis_camera(W=64, H=40, fx=80.0, cx=32.5, cy=20.5)
    op = 0.7
    f = np.array([[1.0, 0.0]])
    sc = scene_from([[0, 0, 2.0]], 0.06, opac=op, feats=f)
    for phi, sig in [(0.5, 0.5), (1.0, 1.0 / (1.0 + math.exp(K * 0.5))), (-1.0, 1.0 / (1.0 + math.exp(-K * 1.5))),
                     (0.0, 1.0 / (1.0 + math.exp(-K * 0.5)))]:
        g = np.array([phi, math.sqrt(max(0.0, 1 - phi * phi))]) * 3.0   # length does not matter
        fgt = np.broadcast_to(g, (40, 64, 2))
        out, _ = _run(sc, cam, {}, fgt)
        assert abs(out["Lgt"][20, 32] - sig * op) < 1e-15
        assert out["Lcf"][20, 32] == 0.0   # one contributor: no pairs
    assert 1.0 / (1.0 + math.exp(K * (0.5 - LAM))) == 0.5


def test_zero_ground_truth_feature_gives_phi_zero():
    cam = axis_camera(W=32, H=32, fx=40.0, cx=16.5, cy=16.5)
    sc = scene_from([[0, 0, 2.0]], 0.06, opac=0.5, feats=[[0.0, 1.0]])
    out, _ = _run(sc, cam, {}, np.zeros((32, 32, 2)))
    assert abs(out["Lgt"][16, 16] - 0.5 / (1.0 + math.exp(-K * LAM))) < 1e-15


def test_two_gaussians_closed_form_nearest_first():
    cam = axis_camera(W=48, H=48, fx=60.0, cx=24.5, cy=24.5)
    fa = _unit([1.0, 0.2, 0.0])
    fb = _unit([0.3, 1.0, 0.5])
    oa, ob = 0.6, 0.45
    # a at depth 2 (near), b at depth 3 (far), both centred on pixel (24, 24)
    sc = scene_from([[0, 0, 2.0], [0, 0, 3.0]], [[0.05] * 3, [0.075] * 3], opac=[oa, ob], feats=[fa, fb])
    gt = _unit([0.9, 0.1, 0.4])
    out, _ = _run(sc, cam, {}, np.broadcast_to(gt, (48, 48, 3)))
    sa = 1.0 / (1.0 + math.exp(K * (fa @ gt - LAM)))
    sb = 1.0 / (1.0 + math.exp(K * (fb @ gt - LAM)))
    assert abs(sa - sb) > 0.1
    w1, w2 = oa, ob * (1 - oa)                       # nearest first
    assert abs(out["Lgt"][24, 24] - (w1 * sa + w2 * sb)) < 1e-14
    assert abs(out["Lcf"][24, 24] - sb * w2 * w1 * (1 - fa @ fb)) < 1e-14
    far_first = sa * (oa * (1 - ob)) * ob * (1 - fa @ fb)
    assert abs(out["Lcf"][24, 24] - far_first) > 1e-3


def test_lgt_equals_render_of_sigma_for_constant_ground_truth():
    sc = small_random_scene(120, seed=21, sh_degree=0, D=6, spread=0.4)
    sc["features"] = _unit(sc["features"])
    cam = axis_camera(W=48, H=40, fx=40.0, t=(0, 0, 2.2))
    gt = np.random.default_rng(3).normal(size=6)
    out, prep = _run(sc, cam, {}, np.broadcast_to(gt, (40, 48, 6)))
    phi = sc["features"] @ gt / np.linalg.norm(gt)
    sig = 1.0 / (1.0 + np.exp(K * (phi - LAM)))
    ren = oracle.forward(sc, [cam], {}, sig[:, None], prep=prep)[0]
    np.testing.assert_allclose(out["Lgt"], ren["feat"][..., 0], rtol=0, atol=1e-13)
    np.testing.assert_allclose(out["W"], 1.0 - ren["T"], rtol=0, atol=1e-13)
    assert np.ptp(sig) > 0.5 and (out["ncontrib"] > 3).mean() > 0.3


def _pairs(sc, cam, prm, prep, fgt, x, y):
    c = oracle.contributors(prep["recs"][0], prep["lists"]["gids"], prep["lists"]["ranges"], cam, prm, x, y)
    f = sc["features"][c["gid"]]
    g = fgt[y, x]
    cos = f @ g / (np.linalg.norm(f, axis=1) * np.linalg.norm(g))
    sig = 1.0 / (1.0 + np.exp(K * (cos - LAM)))
    w = c["alpha"] * c["T"]
    return f, sig, w


def test_linear_recursion_equals_pair_sum():
    sc = small_random_scene(90, seed=22, sh_degree=0, D=5, spread=0.35)
    sc["features"] = _unit(sc["features"])
    cam = axis_camera(W=32, H=28, fx=30.0, t=(0.02, 0, 2.0))
    fgt = np.random.default_rng(4).normal(size=(28, 32, 5))
    out, prep = _run(sc, cam, {}, fgt)
    many = 0
    for y in range(28):
        for x in range(32):
            f, sig, w = _pairs(sc, cam, {}, prep, fgt, x, y)
            n = len(w)
            lcf = 0.0
            for i in range(n):                      # Eq. 6, first line
                for j in range(i):
                    lcf += sig[i] * w[i] * w[j] * (1.0 - float(f[i] @ f[j]))
            lgt = float((w * sig).sum())
            assert abs(out["Lcf"][y, x] - lcf) <= 1e-13
            assert abs(out["Lgt"][y, x] - lgt) <= 1e-13
            assert out["ncontrib"][y, x] == n
            many += n >= 6
    assert many > 100


def test_identical_and_orthogonal_features():
    n = 40
    sc = small_random_scene(n, seed=23, sh_degree=0, D=0, spread=0.3)
    cam = axis_camera(W=32, H=32, fx=30.0, t=(0, 0, 2.0))
    # identical unit features: every pair has 1 - f_i . f_j = 0
    sc["features"] = np.tile(_unit([1.0, 2.0, -1.0, 0.5]), (n, 1))
    fgt = np.random.default_rng(5).normal(size=(32, 32, 4))
    out, _ = _run(sc, cam, {}, fgt)
    assert np.abs(out["Lcf"]).max() < 1e-15 and out["Lgt"].max() > 0.05
    # one-hot (mutually orthogonal) features, f_gt the all-ones vector: a
    # common sigma s and L_cf = s sum_i w_i W_{i-1} = s ((sum w)^2 - sum w^2) / 2
    sc["features"] = np.eye(n)
    fgt = np.ones((32, 32, n))
    out, prep = _run(sc, cam, {}, fgt)
    s = 1.0 / (1.0 + math.exp(K * (1.0 / math.sqrt(n) - LAM)))
    checked = 0
    for y in range(0, 32, 3):
        for x in range(0, 32, 3):
            c = oracle.contributors(prep["recs"][0], prep["lists"]["gids"], prep["lists"]["ranges"], cam, {}, x, y)
            w = c["alpha"] * c["T"]
            want = s * (w.sum() ** 2 - (w * w).sum()) / 2.0
            assert abs(out["Lcf"][y, x] - want) < 1e-14
            assert abs(out["Lgt"][y, x] - s * w.sum()) < 1e-14
            checked += len(w) >= 2
    assert checked > 20


def _ndfd_loss(sc, cam, prm, fgt, a, b):
    out = oracle.ndfd_forward(sc, [cam], prm, sc["features"], [fgt])[0]
    return float((out["Lgt"] * a).sum() + (out["Lcf"] * b).sum())


@pytest.mark.parametrize("seed", [31, 32])
def test_backward_matches_central_differences(seed):
    sc = small_random_scene(12, seed=seed, sh_degree=1, D=4, spread=0.3)
    sc["features"] = _unit(sc["features"])
    sc["opacities"] = np.clip(sc["opacities"], 0.1, 0.9)
    cam = axis_camera(W=28, H=28, fx=26.0, t=(0.02, 0.01, 2.0))
    prm = dict(sh_degree=1)
    g = np.random.default_rng(seed)
    fgt = g.normal(size=(28, 28, 4))
    a, b = g.normal(size=(28, 28)), g.normal(size=(28, 28))
    # pixels with a threshold decision near its edge take no part in the loss,
    # so that the perturbations below flip no decision that matters
    ren = oracle.forward(sc, [cam], prm)[0]
    far = ren["margin"] > 1e-3
    a, b = a * far, b * far
    assert far.mean() > 0.8
    grads = oracle.ndfd_backward(sc, [cam], prm, sc["features"], [fgt], [a], [b])
    assert np.abs(grads["sh"]).max() == 0.0
    checked = 0
    for key in ("means", "scales", "quats", "opacities"):
        base = np.asarray(sc[key], np.float64)
        flat = base.reshape(-1)
        for i in range(flat.size):
            h = 1e-6 * max(1.0, abs(flat[i]))
            vals = []
            for sgn in (1, -1):
                pert = flat.copy()
                pert[i] += sgn * h
                s2 = dict(sc)
                s2[key] = pert.reshape(base.shape)
                vals.append(_ndfd_loss(s2, cam, prm, fgt, a, b))
            fd = (vals[0] - vals[1]) / (2 * h)
            an = grads[key].reshape(-1)[i]
            assert abs(fd - an) <= 2e-6 * max(1.0, abs(fd)), (key, i, fd, an)
            checked += abs(an) > 1e-6
    assert checked > 80


def test_lgt_backward_equals_render_backward_of_sigma():
    sc = small_random_scene(60, seed=24, sh_degree=0, D=5, spread=0.35)
    sc["features"] = _unit(sc["features"])
    cam = axis_camera(W=40, H=36, fx=34.0, t=(0, 0.02, 2.1))
    gt = np.random.default_rng(6).normal(size=5)
    fgt = np.broadcast_to(gt, (36, 40, 5))
    dl = np.random.default_rng(7).normal(size=(36, 40))
    prep = oracle.prepare(sc, [cam], {})
    nd = oracle.ndfd_bwd(prep["recs"][0], sc["features"], prep["lists"]["gids"], prep["lists"]["ranges"], cam, {},
                         (0, 0, 40, 36), fgt, dl, np.zeros_like(dl))
    sig = 1.0 / (1.0 + np.exp(K * (sc["features"] @ gt / np.linalg.norm(gt) - LAM)))
    rb = oracle.render_bwd(prep["recs"][0], sig[:, None], prep["lists"]["gids"], prep["lists"]["ranges"], cam, {},
                           (0, 0, 40, 36), np.zeros((36 * 40, 3)), dl.reshape(-1, 1))
    for k in ("mean2d", "conic", "op"):
        np.testing.assert_allclose(nd[k], rb[k], rtol=0, atol=1e-12 * max(1.0, np.abs(rb[k]).max()))
    assert np.abs(rb["op"]).max() > 1e-2


def test_backward_is_linear_and_sums_over_cameras():
    sc = small_random_scene(30, seed=25, sh_degree=0, D=3, spread=0.4)
    sc["features"] = _unit(sc["features"])
    cams = [axis_camera(W=24, H=24, fx=20.0, t=(0, 0, 2.2)), axis_camera(W=20, H=28, fx=22.0, t=(0.1, 0, 2.0))]
    g = np.random.default_rng(8)
    fg = [g.normal(size=(24, 24, 3)), g.normal(size=(28, 20, 3))]
    a = [g.normal(size=(24, 24)), g.normal(size=(28, 20))]
    b = [g.normal(size=(24, 24)), g.normal(size=(28, 20))]
    z = [np.zeros_like(x) for x in a]
    both = oracle.ndfd_backward(sc, cams, {}, sc["features"], fg, a, b)
    only_gt = oracle.ndfd_backward(sc, cams, {}, sc["features"], fg, a, z)
    only_cf = oracle.ndfd_backward(sc, cams, {}, sc["features"], fg, z, b)
    cam0 = oracle.ndfd_backward(sc, cams[:1], {}, sc["features"], fg[:1], a[:1], b[:1])
    cam1 = oracle.ndfd_backward(sc, cams[1:], {}, sc["features"], fg[1:], a[1:], b[1:])
    for k in ("means", "scales", "quats", "opacities"):
        np.testing.assert_allclose(both[k], only_gt[k] + only_cf[k], atol=1e-12)
        np.testing.assert_allclose(both[k], cam0[k] + cam1[k], atol=1e-12)
        assert np.abs(only_cf[k]).max() > 0
