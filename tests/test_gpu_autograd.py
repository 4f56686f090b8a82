"""The differentiable render (`api.render`, a torch.autograd.Function over
fhgs_render_fwd / fhgs_render_bwd) against the FP64 oracle, on both paths.

`torch.autograd.grad` of sum(dC . rgb + dF . feat) must give the oracle's
gradients of the same scalar (App. A.2 backward plus the projection chain
rule): footprint gradients within 1e-3 relative L2 on both paths; feature
gradients within 1e-4 relative L2 on the FP32 path and 1e-2 on the
tensor-core path, whose feature gradient comes back in the features' dtype
(BF16), a rounding of 2^-9 relative per element on top of the BF16 weights.
The forward outputs equal the Rasterizer's own forward bit for bit.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2505_19154_gb300 import api, synth
from tests.helpers import small_random_scene
from tests.test_gpu_parity import _t, check_grads

pytestmark = pytest.mark.gpu


def _scene(D, bf16):
    sc = small_random_scene(1500, seed=51, sh_degree=2, D=D, spread=0.5)
    sc = {k: (np.asarray(v, np.float32) if isinstance(v, np.ndarray) else v) for k, v in sc.items()}
    if bf16:
        sc["features"] = synth.to_bf16(sc["features"])
    return sc


@pytest.mark.parametrize("path", [api.PATH_FP32, api.PATH_TC])
def test_autograd_render_matches_oracle(path):
    bf16 = path == api.PATH_TC
    D = 128
    sc = _scene(D, bf16)
    cams = [synth.look_at_camera(synth.ring_position(3.0, a, e), w, h)
            for a, e, w, h in [(20, 5, 64, 48), (150, -15, 40, 56)]]
    prm = dict(sh_degree=2, bg=(0.1, 0.3, 0.2))
    P = [c["width"] * c["height"] for c in cams]
    dC, dF = synth.upstream(17, sum(P), D)
    rast = api.Rasterizer(0, sh_degree=2, path=path, bg=prm["bg"])
    leaves = {k: _t(sc[k]).requires_grad_(True) for k in ("means", "scales", "quats", "opacities", "sh")}
    feats = _t(sc["features"], torch.bfloat16 if bf16 else torch.float32).requires_grad_(True)
    rast.ctx.profile(True)
    rgb, feat = api.render(leaves["means"], leaves["scales"], leaves["quats"], leaves["opacities"],
                           leaves["sh"], feats, cams, rast)
    loss = (rgb * _t(dC)).sum() + (feat * _t(dF)).sum()
    names = ("means", "scales", "quats", "opacities", "sh")
    grads = torch.autograd.grad(loss, [leaves[k] for k in names] + [feats])
    torch.cuda.synchronize()
    assert rast.ctx.sync_status() == api.OK
    prof = rast.ctx.profile_read()
    kind = "tc" if bf16 else "fp32"
    assert f"render_fwd_{kind}" in prof and f"render_bwd_{kind}" in prof, prof
    assert grads[-1].dtype == feats.dtype
    got = {k: g.detach().float().cpu().numpy() for k, g in zip(names + ("features",), grads)}

    # the forward is the Rasterizer's, bit for bit
    st = rast.prepare(*(leaves[k].detach() for k in names), cams)
    rgb2, feat2 = rast.forward(st, feats.detach())
    assert torch.equal(rgb.detach(), rgb2) and torch.equal(feat.detach(), feat2)

    prep = oracle.prepare(sc, cams, prm)
    offs = np.cumsum([0] + P)
    ref = oracle.backward(sc, cams, prm, sc["features"], [dC[offs[i]:offs[i + 1]] for i in range(len(cams))],
                          [dF[offs[i]:offs[i + 1]] for i in range(len(cams))], prep=prep)
    check_grads(got, ref, keys=names, tol=1e-3)
    check_grads(got, ref, keys=("features",), tol=1e-2 if bf16 else 1e-4)


def test_autograd_without_feature_grad():
    """Features that do not require a gradient: the backward skips the
    feature-gradient contraction and the footprint gradients are unchanged."""
    sc = _scene(64, True)
    cams = [synth.look_at_camera(synth.ring_position(3.0, 60, 10), 48, 48)]
    dC, dF = synth.upstream(3, 48 * 48, 64)
    rast = api.Rasterizer(0, sh_degree=2, path=api.PATH_TC)
    names = ("means", "scales", "quats", "opacities", "sh")
    leaves = {k: _t(sc[k]).requires_grad_(True) for k in names}
    feats = _t(sc["features"], torch.bfloat16)
    rgb, feat = api.render(*(leaves[k] for k in names), feats, cams, rast)
    loss = (rgb * _t(dC)).sum() + (feat * _t(dF)).sum()
    grads = torch.autograd.grad(loss, [leaves[k] for k in names])
    got = {k: g.cpu().numpy() for k, g in zip(names, grads)}
    ref = oracle.backward(sc, cams, dict(sh_degree=2), sc["features"], [dC], [dF], want_feat=False)
    check_grads(got, ref, keys=names, tol=1e-3)
