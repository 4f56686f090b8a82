"""Oracle of one synthetic training iteration: the loop body of App. A
(Alg. 1, "General Feature Fusion and Densification Framework") with the total
loss of Sec. 3.3,  L = L_rgb + lambda1 L_gt + lambda2 L_cf,  and an Adam
update of the Gaussians' geometry, opacity and colour.

TEST INFRASTRUCTURE ONLY (plain numpy over the FP64 oracle in this package).

Readings, where the paper gives no formula:
  * L_rgb is the L1 photometric loss, the mean of |rendered - target| over
    every pixel and channel of the sampled views (the SSIM term of the 3DGS
    family is left out); d|x|/dx at x = 0 is taken as 0.
  * L_gt and L_cf enter as their means over the same pixels.
  * The optimised (raw) parameters follow the 3DGS family: means, log-scales,
    unnormalised quaternions, opacity logits and SH coefficients; the
    rasterizer sees scales = exp(log-scales) and opacities = sigmoid(logits).
    Features are frozen (Sec. 3.1).
  * Adam (Kingma and Ba): m = b1 m + (1 - b1) g, v = b2 v + (1 - b2) g^2,
    theta -= lr m / (1 - b1^t) / (sqrt(v / (1 - b2^t)) + eps), one learning
    rate per parameter group.
  * Densification is out of scope.
"""
from __future__ import annotations

import numpy as np

from . import backward, forward, ndfd_backward, ndfd_forward, prepare

GROUPS = ("means", "log_scales", "quats", "logit_opacities", "sh")
LR_DEFAULTS = dict(means=1.6e-4, log_scales=5e-3, quats=1e-3, logit_opacities=5e-2, sh=2.5e-3)
ADAM_DEFAULTS = dict(beta1=0.9, beta2=0.999, eps=1e-15)


def raw_from_scene(scene: dict) -> dict:
    op = np.asarray(scene["opacities"], np.float64)
    return dict(means=np.array(scene["means"], np.float64), log_scales=np.log(np.asarray(scene["scales"], np.float64)),
                quats=np.array(scene["quats"], np.float64), logit_opacities=np.log(op / (1.0 - op)),
                sh=np.array(scene["sh"], np.float64))


def scene_from_raw(raw: dict, sh_degree: int, features=None) -> dict:
    s = dict(means=raw["means"], scales=np.exp(raw["log_scales"]), quats=raw["quats"],
             opacities=1.0 / (1.0 + np.exp(-raw["logit_opacities"])), sh=raw["sh"], sh_degree=sh_degree)
    if features is not None:
        s["features"] = features
    return s


def rgb_l1(rgb: np.ndarray, target: np.ndarray, count: int):
    """sum |rgb - target| / count and its gradient with respect to rgb."""
    d = np.asarray(rgb, np.float64) - np.asarray(target, np.float64)
    return float(np.abs(d).sum()) / count, np.sign(d) / count


def loss_and_grads(raw: dict, sh_degree: int, cams: list, targets: list, feats, fgts: list, lam1: float = 1.0,
                   lam2: float = 1.0, params: dict | None = None):
    """The total loss over the views and its gradient with respect to the raw
    parameters.  targets[c]: (H, W, 3); fgts[c]: (H, W, D)."""
    prm = dict(params or {})
    prm["sh_degree"] = sh_degree
    scene = scene_from_raw(raw, sh_degree)
    prep = prepare(scene, cams, prm)
    outs = forward(scene, cams, prm, None, prep=prep)
    npx = sum(int(c["width"]) * int(c["height"]) for c in cams)
    L_rgb, dC = 0.0, []
    for o, tg in zip(outs, targets):
        l, g = rgb_l1(o["rgb"], tg, 3 * npx)
        L_rgb += l
        dC.append(g.reshape(-1, 3))
    nd = ndfd_forward(scene, cams, prm, feats, fgts, prep=prep)
    L_gt = sum(float(r["Lgt"].sum()) for r in nd) / npx
    L_cf = sum(float(r["Lcf"].sum()) for r in nd) / npx
    g_rgb = backward(scene, cams, prm, None, dC, None, prep=prep)
    a = [np.full(int(c["width"]) * int(c["height"]), lam1 / npx) for c in cams]
    b = [np.full(int(c["width"]) * int(c["height"]), lam2 / npx) for c in cams]
    g_nd = ndfd_backward(scene, cams, prm, feats, fgts, a, b, prep=prep)
    g_act = {k: g_rgb[k] + g_nd[k] for k in ("means", "scales", "quats", "opacities", "sh")}
    grads = raw_grads(raw, g_act)
    total = L_rgb + lam1 * L_gt + lam2 * L_cf
    return total, dict(rgb=L_rgb, gt=L_gt, cf=L_cf), grads


def raw_grads(raw: dict, g_act: dict) -> dict:
    """Gradients with respect to the activated values (means, scales, quats,
    opacities, sh) taken to the raw parameters: d/dlog s = s d/ds,
    d/dlogit = op (1 - op) d/dop."""
    s = np.exp(raw["log_scales"])
    op = 1.0 / (1.0 + np.exp(-raw["logit_opacities"]))
    return dict(means=g_act["means"], log_scales=g_act["scales"] * s, quats=g_act["quats"],
                logit_opacities=g_act["opacities"] * op * (1.0 - op), sh=g_act["sh"])


def adam_init(raw: dict) -> dict:
    return {k: (np.zeros_like(raw[k]), np.zeros_like(raw[k])) for k in GROUPS}


def adam_step(raw: dict, grads: dict, state: dict, t: int, lr: dict | None = None, beta1: float = 0.9,
              beta2: float = 0.999, eps: float = 1e-15) -> dict:
    """One Adam update (step number t >= 1); returns the new raw parameters
    and updates `state` in place."""
    lr = dict(LR_DEFAULTS, **(lr or {}))
    out = {}
    for k in GROUPS:
        m, v = state[k]
        g = grads[k]
        m = beta1 * m + (1.0 - beta1) * g
        v = beta2 * v + (1.0 - beta2) * g * g
        state[k] = (m, v)
        mhat = m / (1.0 - beta1 ** t)
        vhat = v / (1.0 - beta2 ** t)
        out[k] = raw[k] - lr[k] * mhat / (np.sqrt(vhat) + eps)
    return out


def train_step(raw: dict, state: dict, t: int, sh_degree: int, cams: list, targets: list, feats, fgts: list,
               lam1: float = 1.0, lam2: float = 1.0, lr: dict | None = None, params: dict | None = None):
    """Loss, gradients and one Adam update: (new raw, total loss, parts)."""
    total, parts, grads = loss_and_grads(raw, sh_degree, cams, targets, feats, fgts, lam1, lam2, params)
    return adam_step(raw, grads, state, t, lr), total, parts
