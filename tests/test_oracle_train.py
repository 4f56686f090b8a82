"""Pins of the training-iteration oracle (App. A, Alg. 1 loop body; the
total loss of Sec. 3.3), no GPU.

(a) Adam's closed forms: the first step moves every parameter by
    -lr g / (|g| + eps); a constant gradient keeps that step size at every
    t (the bias corrections are exact); b1 = b2 = 0 gives the same step from
    any state; a positive rescaling of g leaves the update unchanged;
(b) the L1 loss and its gradient against central differences;
(c) the total loss's raw gradient (through exp and sigmoid) against central
    differences of the whole forward;
(d) a few Adam steps lower the loss of a perturbed scene towards its target.
"""
import numpy as np

import oracle
from oracle import train
from paper_2505_19154_gb300 import synth
from tests.helpers import axis_camera, small_random_scene


def _raw(seed=0):
    g = np.random.default_rng(seed)
    return {k: g.normal(size=(5, 3)) for k in train.GROUPS}


def test_adam_first_step_and_constant_gradient():
    raw = _raw(1)
    g = _raw(2)
    st = train.adam_init(raw)
    lr = {k: 0.01 * (i + 1) for i, k in enumerate(train.GROUPS)}
    eps = 1e-8
    x = raw
    for t in (1, 2, 3, 4):
        y = train.adam_step(x, g, st, t, lr, eps=eps)
        for k in train.GROUPS:
            np.testing.assert_allclose(y[k] - x[k], -lr[k] * g[k] / (np.abs(g[k]) + eps), rtol=1e-12, atol=1e-15)
        x = y


def test_adam_without_memory_and_scale_invariance():
    raw, g1, g2 = _raw(3), _raw(4), _raw(5)
    st = train.adam_init(raw)
    train.adam_step(raw, g1, st, 1)          # some history
    y = train.adam_step(raw, g2, st, 2, beta1=0.0, beta2=0.0, eps=0.0)
    for k in train.GROUPS:
        np.testing.assert_allclose(y[k] - raw[k], -train.LR_DEFAULTS[k] * np.sign(g2[k]), rtol=1e-12, atol=1e-15)
    s1, s2 = train.adam_init(raw), train.adam_init(raw)
    a = b = raw
    for t, gg in enumerate((g1, g2, g1), start=1):
        a = train.adam_step(a, gg, s1, t, eps=0.0)
        b = train.adam_step(b, {k: 7.5 * v for k, v in gg.items()}, s2, t, eps=0.0)
    for k in train.GROUPS:
        np.testing.assert_allclose(a[k], b[k], rtol=1e-12, atol=1e-14)


def test_l1_loss_gradient():
    g = np.random.default_rng(6)
    x, y = g.normal(size=(4, 5, 3)), g.normal(size=(4, 5, 3))
    L, d = train.rgb_l1(x, y, 60)
    assert abs(L - np.abs(x - y).mean()) < 1e-15
    for idx in [(0, 0, 0), (3, 4, 2), (2, 1, 1)]:
        e = np.zeros_like(x)
        e[idx] = 1e-7
        fd = (train.rgb_l1(x + e, y, 60)[0] - train.rgb_l1(x - e, y, 60)[0]) / 2e-7
        assert abs(fd - d[idx]) < 1e-7


def _case():
    sc = small_random_scene(10, seed=41, sh_degree=1, D=0, spread=0.3)
    sc["opacities"] = np.clip(sc["opacities"], 0.1, 0.9)
    sc["quats"] = sc["quats"] / np.linalg.norm(sc["quats"], axis=1, keepdims=True)
    cams = [axis_camera(W=24, H=20, fx=22.0, t=(0.02, 0.01, 2.0)), axis_camera(W=20, H=24, fx=20.0, t=(-0.05, 0, 2.1))]
    protos = synth.ndfd_prototypes(41, 4)
    feats = synth.ndfd_features(41, 10, protos).astype(np.float64)
    fgts = [synth.ndfd_ground_truth(41, v, c["height"], c["width"], protos, block=6) for v, c in enumerate(cams)]
    g = np.random.default_rng(9)
    # targets 0.3 away from the render in a random direction: no |.| kink is near
    outs = oracle.forward(sc, cams, dict(sh_degree=1))
    targets = [o["rgb"] + 0.3 * np.sign(g.normal(size=o["rgb"].shape)) for o in outs]
    return sc, cams, feats, fgts, targets


def test_total_loss_gradient_matches_central_differences():
    sc, cams, feats, fgts, targets = _case()
    raw = train.raw_from_scene(sc)
    lam1, lam2 = 0.7, 1.3
    L0, parts, grads = train.loss_and_grads(raw, 1, cams, targets, feats, fgts, lam1, lam2)
    assert parts["gt"] > 0 and parts["cf"] > 0
    checked = 0
    for k in train.GROUPS:
        flat = raw[k].reshape(-1)
        for i in range(flat.size):
            fds = []
            for h in (1e-6, 5e-7):
                vals = []
                for sgn in (1, -1):
                    r2 = {kk: vv.copy() for kk, vv in raw.items()}
                    r2[k].reshape(-1)[i] += sgn * h
                    vals.append(train.loss_and_grads(r2, 1, cams, targets, feats, fgts, lam1, lam2)[0])
                fds.append((vals[0] - vals[1]) / (2 * h))
            if abs(fds[0] - fds[1]) > 1e-6 * max(1.0, abs(fds[0])):
                continue   # a contribute/skip decision flipped inside the step
            an = grads[k].reshape(-1)[i]
            assert abs(fds[0] - an) <= 2e-6 * max(1.0, abs(fds[0])), (k, i, fds[0], an)
            checked += abs(an) > 1e-8
    assert checked > 60


def test_adam_steps_lower_the_loss():
    sc, cams, feats, fgts, _ = _case()
    targets = [o["rgb"] for o in oracle.forward(sc, cams, dict(sh_degree=1))]
    raw = train.raw_from_scene(sc)
    g = np.random.default_rng(3)
    raw["means"] = raw["means"] + 0.02 * g.normal(size=raw["means"].shape)
    raw["sh"] = raw["sh"] + 0.2 * g.normal(size=raw["sh"].shape)
    st = train.adam_init(raw)
    lr = dict(means=2e-3, log_scales=1e-2, quats=1e-2, logit_opacities=5e-2, sh=2e-2)
    losses = []
    for t in range(1, 13):
        raw, L, parts = train.train_step(raw, st, t, 1, cams, targets, feats, fgts, 0.0, 0.0, lr)
        losses.append(parts["rgb"])
    assert losses[-1] < 0.6 * losses[0], losses
