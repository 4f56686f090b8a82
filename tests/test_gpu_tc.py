"""Parity of the tcgen05 tensor-core path against the FP64 oracle.

Bars: RGB within 1e-5 max abs and `last` exact (the weights are the FP32
ones); features within 1e-2 of max|F| (the BF16 feature path: weights are
rounded to BF16, relative error <= 2^-9 per term); footprint gradients
(means, scales, quats, opacities, SH) within 1e-3 relative L2 (dL/dF enters
the dF.Fe^T contraction as BF16 hi + lo, ~16 mantissa bits); feature
gradients within 1e-2 relative L2 (BF16 weights).  Features are BF16 inputs,
so the oracle uses exactly the same feature values.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2505_19154_gb300 import api, synth
from tests.helpers import small_random_scene
from tests.test_gpu_parity import _t, check_grads, check_image

pytestmark = pytest.mark.gpu


def run_tc(scene, cams, prm, d_split=0, dC=None, dF=None):
    rast = api.Rasterizer(0, sh_degree=prm.get("sh_degree", 0), path=api.PATH_TC,
                          bg=prm.get("bg", (0.0, 0.0, 0.0)), d_split=d_split)
    t = {k: _t(scene[k]) for k in ("means", "scales", "quats", "opacities", "sh")}
    feats = _t(scene["features"], torch.bfloat16)
    rast.ctx.profile(True)
    st = rast.prepare(t["means"], t["scales"], t["quats"], t["opacities"], t["sh"], cams)
    rgb, feat = rast.forward(st, feats)
    out = dict(rgb=rgb.cpu().numpy(), feat=feat.cpu().numpy(), T=st["T"].cpu().numpy(),
               last=st["last"].cpu().numpy())
    if dC is not None:
        g = rast.backward(st, _t(dC), None if dF is None else _t(dF))
        out["grads"] = {k: (None if v is None else v.cpu().numpy()) for k, v in g.items()}
    torch.cuda.synchronize()
    assert rast.ctx.sync_status() == api.OK
    prof = rast.ctx.profile_read()
    assert "render_fwd_tc" in prof, prof
    if dC is not None:
        assert "render_bwd_tc" in prof, prof
    return out


def bf16_scene(n, seed, D, sh_degree=1, spread=0.5):
    sc = small_random_scene(n, seed=seed, sh_degree=sh_degree, D=D, spread=spread)
    sc = {k: (np.asarray(v, np.float32) if isinstance(v, np.ndarray) else v) for k, v in sc.items()}
    sc["features"] = synth.to_bf16(sc["features"])
    return sc


@pytest.mark.parametrize("d_split", [64, 128])
def test_tc_forward_small(d_split):
    sc = bf16_scene(600, seed=41, D=128)
    cams = [synth.look_at_camera(synth.ring_position(3.0, 10, 5), 48, 40)]
    prm = dict(sh_degree=1)
    prep = oracle.prepare(sc, cams, prm)
    out = run_tc(sc, cams, prm, d_split=d_split)
    refs = oracle.forward(sc, cams, prm, sc["features"], prep=prep)
    check_image(out, refs, cams, feat_tol=1e-2)


def test_tc_forward_multicamera_ragged_dsplit256():
    sc = bf16_scene(4000, seed=42, D=256, sh_degree=2)
    cams = [synth.look_at_camera(synth.ring_position(3.0, a, e), w, h)
            for a, e, w, h in [(0, 0, 70, 50), (130, 20, 33, 47), (250, -25, 96, 64)]]
    prm = dict(sh_degree=2, bg=(0.1, 0.2, 0.3))
    prep = oracle.prepare(sc, cams, prm)
    out = run_tc(sc, cams, prm, d_split=256)
    refs = oracle.forward(sc, cams, prm, sc["features"], prep=prep)
    check_image(out, refs, cams, feat_tol=1e-2)


@pytest.mark.parametrize("d_split", [64, 128, 256])
def test_tc_backward_small(d_split):
    sc = bf16_scene(1500, seed=43, D=256, sh_degree=3)
    cams = [synth.look_at_camera(synth.ring_position(3.0, 30, 10), 64, 48)]
    prm = dict(sh_degree=3, bg=(0.2, 0.1, 0.3))
    dC, dF = synth.upstream(9, 64 * 48, 256)
    prep = oracle.prepare(sc, cams, prm)
    out = run_tc(sc, cams, prm, d_split=d_split, dC=dC, dF=dF)
    refs = oracle.forward(sc, cams, prm, sc["features"], prep=prep)
    check_image(out, refs, cams, feat_tol=1e-2)
    ref = oracle.backward(sc, cams, prm, sc["features"], [dC], [dF], prep=prep)
    check_grads(out["grads"], ref, keys=("means", "scales", "quats", "opacities", "sh"), tol=1e-3)
    check_grads(out["grads"], ref, keys=("features",), tol=1e-2)


def test_tc_backward_without_feature_upstream():
    """grad_feat NULL with grad_features requested: the tensor-core backward
    stages no dL/dF (zero), so the footprint gradients are the colour-only
    ones and the feature gradient is exactly zero."""
    sc = bf16_scene(1200, seed=47, D=256, sh_degree=2)
    cams = [synth.look_at_camera(synth.ring_position(3.0, 200, -15), 80, 56)]
    prm = dict(sh_degree=2, bg=(0.3, 0.1, 0.2))
    dC, _ = synth.upstream(4, 80 * 56, 256)
    prep = oracle.prepare(sc, cams, prm)
    out = run_tc(sc, cams, prm, dC=dC, dF=None)
    assert out["grads"]["features"] is not None and not np.any(out["grads"]["features"])
    ref = oracle.backward(sc, cams, prm, sc["features"], [dC], [np.zeros((80 * 56, 256))], prep=prep)
    check_grads(out["grads"], ref, keys=("means", "scales", "quats", "opacities", "sh"), tol=1e-3)


@pytest.mark.slow
def test_tc_config2_forward_backward():
    scene, cams = synth.config2(0)
    scene["features"] = synth.to_bf16(scene["features"])
    prm = dict(sh_degree=3)
    dC, dF = synth.upstream(2, 512 * 512, 128)
    prep = oracle.prepare(scene, cams, prm)
    out = run_tc(scene, cams, prm, dC=dC, dF=dF)
    refs = oracle.forward(scene, cams, prm, scene["features"], prep=prep)
    check_image(out, refs, cams, feat_tol=1e-2)
    ref = oracle.backward(scene, cams, prm, scene["features"], [dC], [dF], prep=prep)
    check_grads(out["grads"], ref, keys=("means", "scales", "quats", "opacities", "sh"), tol=1e-3)
    check_grads(out["grads"], ref, keys=("features",), tol=1e-2)


@pytest.mark.parametrize("D", [128, 192])
def test_tc_fusion_small_against_oracle_and_fp32_path(D):
    """Tensor-core fusion (one D slice at 128, three at 192) against the
    oracle composited over the FP32 specification's footprints, with the
    fusion margin rule; and against the FP32 CUDA-core fusion.  The maps are
    unit-norm per pixel (the workload's recipe): a weight change d at pixel p
    moves num/den by d (f_p - out) / den, at most 2 d / den when |f_p| = 1,
    which is what the margin rule's allowance 2 wflip / (den |out|) assumes."""
    sc = small_random_scene(2500, seed=33, sh_degree=1, D=0, spread=0.5)
    sc = {k: (np.asarray(v, np.float32) if isinstance(v, np.ndarray) else v) for k, v in sc.items()}
    views = [synth.look_at_camera(synth.ring_position(3.0, a, e), w, h)
             for a, e, w, h in [(10, 5, 80, 48), (130, -10, 64, 72), (250, 20, 50, 40)]]
    prm = dict(sh_degree=1)
    maps = [synth.smooth_feature_map(4, i, v["height"], v["width"], D) for i, v in enumerate(views)]
    prep = oracle.prepare(sc, views, prm, geometry="fp32")
    ref = oracle.fuse(sc, views, maps, prm, prep=prep)
    t = {k: _t(sc[k]) for k in ("means", "scales", "quats", "opacities", "sh")}
    dmaps = [_t(m).view(-1, D) for m in maps]
    outs = {}
    for path, cut in ((api.PATH_TC, 0), (api.PATH_TC, 1), (api.PATH_FP32, 0)):
        rast = api.Rasterizer(0, sh_degree=1, path=path, list_cut=cut)
        rast.ctx.profile(True)
        o, n_, d_ = rast.fuse(t["means"], t["scales"], t["quats"], t["opacities"], t["sh"], views, dmaps)
        torch.cuda.synchronize()
        assert rast.ctx.sync_status() == api.OK
        prof = rast.ctx.profile_read()
        assert ("fuse_tc" if path == api.PATH_TC else "fuse_fp32") in prof, prof
        outs[(path, cut)] = (o.cpu().numpy().astype(np.float64), d_.cpu().numpy().astype(np.float64))
    seen = ref["den"] > 1e-6
    assert seen.sum() > 300
    fn = np.maximum(np.linalg.norm(ref["out"], axis=1), 1e-30)
    risk = 2.0 * ref["wflip"] / np.maximum(ref["den"], 1e-30) / fn
    for path, (o, d_) in outs.items():
        rel = np.linalg.norm(o - ref["out"], axis=1) / fn
        chk = seen & (risk <= 1e-4)
        print(f"fusion {path}: {int((seen & ~chk).sum())} of {int(seen.sum())} seen Gaussians near a threshold")
        assert (seen & ~chk).sum() <= 0.06 * seen.sum()
        assert rel[chk].max() <= 1e-4, (path, rel[chk].max())
        assert np.all(rel[seen] <= 1e-4 + risk[seen]), path
        assert np.abs(d_ - ref["den"]).max() <= 1e-4 * max(1.0, ref["den"].max()), path
        assert np.all(o[ref["den"] == 0] == 0), path


def test_fusion_view_groups_against_oracle_and_single_views():
    """Eleven ragged views fuse in two groups (8 + 3 views, one projection,
    binning and fusion launch each): against the oracle with the fusion
    margin rule, and against the same views fused one call per view (the
    same weights, so num and den differ only by the order of their float
    additions).  Unit-norm smooth maps, as in the small fusion test above."""
    D = 64
    sc = small_random_scene(2500, seed=35, sh_degree=1, D=0, spread=0.5)
    sc = {k: (np.asarray(v, np.float32) if isinstance(v, np.ndarray) else v) for k, v in sc.items()}
    spec = [(33 * i, (-20, 0, 15, 25)[i % 4], (48, 64, 40, 72)[i % 4], (40, 56, 64, 36)[i % 3]) for i in range(11)]
    views = [synth.look_at_camera(synth.ring_position(3.0, a, e), w, h) for a, e, w, h in spec]
    prm = dict(sh_degree=1)
    maps = [synth.smooth_feature_map(5, i, v["height"], v["width"], D) for i, v in enumerate(views)]
    prep = oracle.prepare(sc, views, prm, geometry="fp32")
    ref = oracle.fuse(sc, views, maps, prm, prep=prep)
    t = {k: _t(sc[k]) for k in ("means", "scales", "quats", "opacities", "sh")}
    gs = tuple(t[k] for k in ("means", "scales", "quats", "opacities", "sh"))
    dmaps = [_t(m).view(-1, D) for m in maps]
    seen = ref["den"] > 1e-6
    assert seen.sum() > 300
    fn = np.maximum(np.linalg.norm(ref["out"], axis=1), 1e-30)
    risk = 2.0 * ref["wflip"] / np.maximum(ref["den"], 1e-30) / fn
    for path, cut in ((api.PATH_TC, 1), (api.PATH_FP32, 0)):
        rast = api.Rasterizer(0, sh_degree=1, path=path, list_cut=cut)
        rast.ctx.profile(True)
        o, num, den = rast.fuse(*gs, views, dmaps)
        torch.cuda.synchronize()
        assert rast.ctx.sync_status() == api.OK
        prof = rast.ctx.profile_read()
        name = "fuse_tc" if path == api.PATH_TC else "fuse_fp32"
        assert prof[name][0] == 2 and prof["fuse_bin_sort"][0] >= 2, prof  # two groups
        o = o.cpu().numpy().astype(np.float64)
        d_ = den.cpu().numpy().astype(np.float64)
        rel = np.linalg.norm(o - ref["out"], axis=1) / fn
        chk = seen & (risk <= 1e-4)
        assert (seen & ~chk).sum() <= 0.06 * seen.sum()
        assert rel[chk].max() <= 1e-4, (path, rel[chk].max())
        assert np.all(rel[seen] <= 1e-4 + risk[seen]), path
        assert np.abs(d_ - ref["den"]).max() <= 1e-4 * max(1.0, ref["den"].max()), path
        assert np.all(o[ref["den"] == 0] == 0), path
        # one call per view into the same accumulators
        num1 = torch.zeros_like(num)
        den1 = torch.zeros_like(den)
        for v, m in zip(views, dmaps):
            rast.fuse_accumulate(gs, [v], [m], num1, den1)
        torch.cuda.synchronize()
        n0, n1 = num.cpu().numpy().astype(np.float64), num1.cpu().numpy().astype(np.float64)
        d0, d1 = den.cpu().numpy().astype(np.float64), den1.cpu().numpy().astype(np.float64)
        assert np.array_equal(d0 > 0, d1 > 0), path
        assert np.abs(d0 - d1).max() <= 1e-5 * max(1.0, d0.max()), path
        nrm = np.maximum(np.linalg.norm(n0, axis=1), 1e-30)
        assert (np.linalg.norm(n0 - n1, axis=1) / nrm)[d0 > 0].max() <= 1e-5, path


@pytest.mark.parametrize("D,cams_spec", [(256, [(30, 10, 64, 48)]),
                                         (384, [(0, 0, 70, 50), (130, 20, 33, 47), (250, -25, 96, 64)]),
                                         (128, [(200, 15, 80, 56)])])
def test_tc_backward_streamed(D, cams_spec):
    """The streamed backward (d_split 1: dL/dF in 64-channel chunks, one
    scalar pass per batch over all D channels) against the oracle: one
    camera at D = 256, three ragged cameras at D = 384 (three 128-channel
    feature-gradient blocks per batch), D = 128 (one block)."""
    sc = bf16_scene(1500, seed=44 + D, D=D, sh_degree=3)
    cams = [synth.look_at_camera(synth.ring_position(3.0, a, e), w, h) for a, e, w, h in cams_spec]
    prm = dict(sh_degree=3, bg=(0.2, 0.1, 0.3))
    P = sum(c["width"] * c["height"] for c in cams)
    dC, dF = synth.upstream(10 + D, P, D)
    prep = oracle.prepare(sc, cams, prm)
    out = run_tc(sc, cams, prm, d_split=1, dC=dC, dF=dF)
    refs = oracle.forward(sc, cams, prm, sc["features"], prep=prep)
    check_image(out, refs, cams, feat_tol=1e-2)
    offs = np.cumsum([0] + [c["width"] * c["height"] for c in cams])
    ref = oracle.backward(sc, cams, prm, sc["features"], [dC[offs[i]:offs[i + 1]] for i in range(len(cams))],
                          [dF[offs[i]:offs[i + 1]] for i in range(len(cams))], prep=prep)
    check_grads(out["grads"], ref, keys=("means", "scales", "quats", "opacities", "sh"), tol=1e-3)
    check_grads(out["grads"], ref, keys=("features",), tol=1e-2)


def test_tc_backward_streamed_without_feature_gradient():
    """grad_features not requested: the streamed kernel still computes G for
    dL/dw and issues no feature-gradient MMA."""
    sc = bf16_scene(1200, seed=48, D=256, sh_degree=2)
    cams = [synth.look_at_camera(synth.ring_position(3.0, 100, -5), 72, 40)]
    prm = dict(sh_degree=2)
    dC, dF = synth.upstream(21, 72 * 40, 256)
    rast = api.Rasterizer(0, sh_degree=2, path=api.PATH_TC, d_split=1)
    t = {k: _t(sc[k]) for k in ("means", "scales", "quats", "opacities", "sh")}
    st = rast.prepare(t["means"], t["scales"], t["quats"], t["opacities"], t["sh"], cams)
    rast.forward(st, _t(sc["features"], torch.bfloat16))
    g = rast.backward(st, _t(dC), _t(dF), want_feat_grad=False)
    torch.cuda.synchronize()
    assert rast.ctx.sync_status() == api.OK
    assert g.get("features") is None
    ref = oracle.backward(sc, cams, prm, sc["features"], [dC], [dF], want_feat=False)
    got = {k: v.cpu().numpy() for k, v in g.items() if v is not None}
    check_grads(got, ref, keys=("means", "scales", "quats", "opacities", "sh"), tol=1e-3)
