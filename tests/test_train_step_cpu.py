"""The training-iteration host code (paper_2505_19154_gb300.train.TrainStep)
on a backend built from the oracle (no GPU): its sequencing must give
exactly the oracle's own iteration (oracle/train.py) step after step."""
import numpy as np

import oracle
from oracle import train as otrain
from paper_2505_19154_gb300 import synth
from paper_2505_19154_gb300.train import GROUPS, TrainStep
from tests.helpers import axis_camera, small_random_scene


class OracleBackend:
    def __init__(self, sh_degree):
        self.prm = dict(sh_degree=sh_degree)

    def adam_init(self, raw, sh_degree):
        return otrain.adam_init(raw)

    def activate(self, raw):
        return dict(scales=np.exp(raw["log_scales"]), opacities=1.0 / (1.0 + np.exp(-raw["logit_opacities"])))

    def prepare(self, params, cam):
        scene = dict(params, sh_degree=self.prm["sh_degree"])
        return dict(scene=scene, cam=cam, prep=oracle.prepare(scene, [cam], self.prm))

    def render(self, st):
        return oracle.forward(st["scene"], [st["cam"]], self.prm, None, prep=st["prep"])[0]["rgb"].reshape(-1, 3)

    def l1(self, rgb, target):
        return otrain.rgb_l1(rgb, np.asarray(target).reshape(rgb.shape), rgb.size)

    def ndfd(self, st, features, feat_gt):
        r = oracle.ndfd_forward(st["scene"], [st["cam"]], self.prm, features, [feat_gt], prep=st["prep"])[0]
        return r["Lgt"], r["Lcf"]

    def total(self, x):
        return float(np.sum(x))

    def backward(self, st, grad_rgb):
        return oracle.backward(st["scene"], [st["cam"]], self.prm, None, [grad_rgb], None, prep=st["prep"])

    def ndfd_backward(self, st, features, feat_gt, a, b):
        P = int(st["cam"]["width"]) * int(st["cam"]["height"])
        return oracle.ndfd_backward(st["scene"], [st["cam"]], self.prm, features, [feat_gt], [np.full(P, a)],
                                    [np.full(P, b)], prep=st["prep"])

    def add(self, g1, g2):
        return {k: g1[k] + g2[k] for k in ("means", "scales", "quats", "opacities", "sh")}

    def adam(self, raw, grads, state, t, lr, beta1, beta2, eps):
        new = otrain.adam_step(raw, otrain.raw_grads(raw, grads), state, t, dict(zip(GROUPS, lr)), beta1, beta2, eps)
        for k in GROUPS:
            raw[k][...] = new[k]
        return self.activate(raw)


def test_train_step_sequencing_equals_the_oracle_iteration():
    sc = small_random_scene(12, seed=51, sh_degree=1, D=0, spread=0.3)
    sc["opacities"] = np.clip(sc["opacities"], 0.1, 0.9)
    cam = axis_camera(W=22, H=20, fx=21.0, t=(0.01, 0.02, 2.0))
    protos = synth.ndfd_prototypes(51, 4)
    feats = synth.ndfd_features(51, 12, protos).astype(np.float64)
    fgt = synth.ndfd_ground_truth(51, 0, 20, 22, protos, block=5)
    target = oracle.forward(sc, [cam], dict(sh_degree=1))[0]["rgb"] + 0.05
    raw0 = otrain.raw_from_scene(sc)
    lr = (2e-3, 1e-2, 1e-2, 5e-2, 2e-2)
    step = TrainStep(OracleBackend(1), {k: v.copy() for k, v in raw0.items()}, 1, feats, lr=lr, lam1=0.7, lam2=1.3)
    ref_raw = {k: v.copy() for k, v in raw0.items()}
    ref_state = otrain.adam_init(ref_raw)
    for t in (1, 2, 3):
        got = step(cam, target, fgt)
        ref_raw, total, parts = otrain.train_step(ref_raw, ref_state, t, 1, [cam], [target], feats, [fgt], 0.7, 1.3,
                                                  dict(zip(GROUPS, lr)))
        assert abs(got["total"] - total) < 1e-12 and abs(got["cf"] - parts["cf"]) < 1e-12
        for k in GROUPS:
            np.testing.assert_allclose(step.raw[k], ref_raw[k], rtol=0, atol=1e-12, err_msg=k)
    assert parts["gt"] > 0 and parts["cf"] > 0
