"""Parity of the 2DGS surfel path (Sec. 3.1, Eq. 1-3; FHGS_GEOM_SURFEL)
against the FP64 oracle, through the C ABI.

Bars: tile keys, ids and ranges bit-exact against the oracle's binary32
surfel binning rule; RGB and T within 5e-5 max abs and features within
1e-4 x max(1, max|F|) outside margin pixels (the margin rule of the EWA
path: decisions that settle a pixel's contributor set within 1e-5 of their
threshold, capped at 0.1 % of the pixels plus a few); gradients of means,
(s_u, s_v), quaternions, opacities, SH and features within 1e-3 relative L2
(FP32 against FP64, as for the EWA path).  The colour bar is five times the
EWA path's: the FP32 pixel offset from the projected centre carries a
rounding of up to half an ulp of the pixel coordinate, and u, v move by
that over the surfel's thinnest screen extent, which has no floor (a surfel
seen nearly edge-on is arbitrarily thin; the EWA footprint has the 0.3 px^2
dilation).  Measured: 1.07e-5 worst in the 33 px wide camera below.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2505_19154_gb300 import api, synth
from tests.helpers import MARGIN_TOL, check_margin_count
from tests.test_gpu_parity import _t, check_grads

pytestmark = pytest.mark.gpu


def surfel_scene(n, seed, sh_degree, D, spread=0.45):
    g = synth.rng(seed, 93)
    q = g.normal(0.0, 1.0, (n, 4))
    s = dict(means=g.normal(0.0, spread, (n, 3)), scales=np.exp(g.uniform(-3.2, -1.9, (n, 3))), quats=q,
             opacities=1.0 / (1.0 + np.exp(-g.normal(0.0, 1.0, n))),
             sh=g.normal(0.0, 0.3, (n, (sh_degree + 1) ** 2, 3)), sh_degree=sh_degree)
    s["sh"][:, 0, :] += 0.5
    if D:
        s["features"] = g.normal(0.0, 1.0, (n, D))
    # binary32 inputs, as the kernels read them
    s = {k: (np.asarray(v, np.float32).astype(np.float64) if isinstance(v, np.ndarray) else v) for k, v in s.items()}
    s["scales2"] = s["scales"][:, :2].copy()
    return s


def run_surfel(scene, cams, prm, dC=None, dF=None):
    rast = api.Rasterizer(0, sh_degree=prm["sh_degree"], path=api.PATH_FP32, bg=prm.get("bg", (0.0, 0.0, 0.0)),
                          keep_keys=True, geometry=api.GEOM_SURFEL)
    t = {k: _t(scene[k]) for k in ("means", "scales", "quats", "opacities", "sh")}
    feats = _t(scene["features"]) if scene.get("features") is not None else None
    rast.ctx.profile(True)
    st = rast.prepare(t["means"], t["scales"], t["quats"], t["opacities"], t["sh"], cams)
    rgb, feat = rast.forward(st, feats)
    out = dict(rgb=rgb.cpu().numpy(), feat=None if feat is None else feat.cpu().numpy(), T=st["T"].cpu().numpy(),
               count=st["n_instances"])
    n = out["count"]
    out["keys"] = st["keys"][:n].cpu().numpy().view(np.uint64)
    out["gids"] = st["gids"][:n].cpu().numpy().view(np.uint32)
    out["ranges"] = st["ranges"].cpu().numpy().view(np.uint32)
    if dC is not None:
        g = rast.backward(st, _t(dC), None if dF is None else _t(dF))
        out["grads"] = {k: (None if v is None else v.cpu().numpy()) for k, v in g.items()}
    torch.cuda.synchronize()
    assert rast.ctx.sync_status() == api.OK
    prof = rast.ctx.profile_read()
    assert "render_fwd_surfel" in prof, prof
    if dC is not None:
        assert "render_bwd_surfel" in prof, prof
    return out


def oracle_lists(scene, cams, prm):
    bins = [oracle.bin_surfel_f32(np.asarray(scene["means"], np.float32), np.asarray(scene["quats"], np.float32),
                                  np.asarray(scene["scales2"], np.float32), c, prm) for c in cams]
    return oracle.tile_lists(bins, cams, prm)


def check_surfel_image(out, scene, cams, prm, feat_tol=1e-4):
    off = n_margin = n_pix = 0
    for cam in cams:
        P = cam["width"] * cam["height"]
        ref = oracle.surfel_forward(scene, cam, prm, feats=scene.get("features"))
        ok = ref["margin"].reshape(-1) > MARGIN_TOL
        n_margin += int((~ok).sum())
        n_pix += P
        e_rgb = np.abs(out["rgb"][off:off + P] - ref["rgb"].reshape(-1, 3))[ok].max(initial=0)
        e_T = np.abs(out["T"][off:off + P] - ref["T"].reshape(-1))[ok].max(initial=0)
        print(f"surfel camera {cam['width']}x{cam['height']}: rgb err {e_rgb:.3g}, T err {e_T:.3g}")
        assert e_rgb <= 5e-5 and e_T <= 5e-5, (e_rgb, e_T)
        if ref["feat"] is not None and out["feat"] is not None:
            D = ref["feat"].shape[-1]
            fr = ref["feat"].reshape(-1, D)
            err = np.abs(out["feat"][off:off + P] - fr)[ok].max(initial=0) / max(1.0, np.abs(fr).max())
            assert err <= feat_tol, err
        assert (ref["ncontrib"] > 2).mean() > 0.1   # the scene really overlaps
        off += P
    check_margin_count(n_margin, n_pix, "surfel image")


def surfel_ref_grads(scene, cams, prm, dC, dF):
    P = [c["width"] * c["height"] for c in cams]
    offs = np.cumsum([0] + P)
    tot = None
    for i, cam in enumerate(cams):
        g = oracle.surfel_backward(scene, cam, prm, dC[offs[i]:offs[i + 1]], feats=scene.get("features"),
                                   dF=None if dF is None else dF[offs[i]:offs[i + 1]])
        tot = g if tot is None else {k: (None if v is None else v + g[k]) for k, v in tot.items()}
    return tot


def test_surfel_lists_image_and_gradients_single_camera():
    sc = surfel_scene(900, seed=3, sh_degree=1, D=16)
    cams = [synth.look_at_camera(synth.ring_position(2.6, 20, 10), 72, 56)]
    prm = dict(sh_degree=1, bg=(0.1, 0.2, 0.3))
    dC, dF = synth.upstream(12, 72 * 56, 16)
    out = run_surfel(sc, cams, prm, dC=dC, dF=dF)
    L = oracle_lists(sc, cams, prm)
    assert out["count"] == len(L["keys"]) and out["count"] > 1000
    np.testing.assert_array_equal(out["keys"], L["keys"])
    np.testing.assert_array_equal(out["gids"], L["gids"])
    np.testing.assert_array_equal(out["ranges"], L["ranges"])
    check_surfel_image(out, sc, cams, prm)
    ref = surfel_ref_grads(sc, cams, prm, dC, dF)
    got = dict(out["grads"])
    assert np.all(got["scales"][:, 2] == 0.0)
    got["scales2"] = got["scales"][:, :2]
    check_grads(got, ref, keys=("means", "scales2", "quats", "opacities", "sh", "features"), tol=1e-3)


def test_surfel_ragged_multicamera_sh3():
    sc = surfel_scene(2500, seed=4, sh_degree=3, D=0, spread=0.5)
    cams = [synth.look_at_camera(synth.ring_position(3.0, a, e), w, h)
            for a, e, w, h in [(0, 0, 70, 50), (40, 20, 33, 47), (200, -25, 96, 64)]]
    prm = dict(sh_degree=3)
    P = sum(c["width"] * c["height"] for c in cams)
    dC, _ = synth.upstream(13, P, 8)
    out = run_surfel(sc, cams, prm, dC=dC)
    L = oracle_lists(sc, cams, prm)
    np.testing.assert_array_equal(out["keys"], L["keys"])
    np.testing.assert_array_equal(out["gids"], L["gids"])
    np.testing.assert_array_equal(out["ranges"], L["ranges"])
    check_surfel_image(out, sc, cams, prm)
    ref = surfel_ref_grads(sc, cams, prm, dC, None)
    got = dict(out["grads"])
    got["scales2"] = got["scales"][:, :2]
    check_grads(got, ref, keys=("means", "scales2", "quats", "opacities", "sh"), tol=1e-3)


def test_surfel_tensor_core_forward_and_backward():
    """BF16 features: FHGS_PATH_AUTO renders surfels on the tensor cores (the
    same surfel weights, BF16 weights in the blend: features within 1e-2 of
    max|F|, the EWA tensor-core bar) and runs the tensor-core backward (the
    footprint chain per (pixel, surfel) on the CUDA cores): geometry
    gradients within 1e-3, feature gradients within 1e-2 (BF16 weights), the
    EWA tensor-core bars.  The FP32 path still renders and differentiates the
    same scene within the FP32 bars; fusion is refused before any launch."""
    sc = surfel_scene(1500, seed=5, sh_degree=1, D=256, spread=0.45)
    sc["features"] = synth.to_bf16(sc["features"])
    cams = [synth.look_at_camera(synth.ring_position(2.6, a, e), w, h)
            for a, e, w, h in [(120, -10, 48, 40), (300, 15, 70, 52)]]
    prm = dict(sh_degree=1)
    P = sum(c["width"] * c["height"] for c in cams)
    dC, dF = synth.upstream(21, P, 256)
    rast = api.Rasterizer(0, sh_degree=1, geometry=api.GEOM_SURFEL)
    t = {k: _t(sc[k]) for k in ("means", "scales", "quats", "opacities", "sh")}
    rast.ctx.profile(True)
    st = rast.prepare(t["means"], t["scales"], t["quats"], t["opacities"], t["sh"], cams)
    feats = _t(sc["features"], torch.bfloat16)
    rgb, feat = rast.forward(st, feats)
    g = rast.backward(st, _t(dC), _t(dF))
    torch.cuda.synchronize()
    assert rast.ctx.sync_status() == api.OK
    prof = rast.ctx.profile_read()
    assert "render_fwd_tc_surfel" in prof and "render_bwd_tc_surfel" in prof, prof
    check_surfel_image(dict(rgb=rgb.cpu().numpy(), feat=feat.cpu().numpy(), T=st["T"].cpu().numpy()), sc, cams, prm,
                       feat_tol=1e-2)
    ref = surfel_ref_grads(sc, cams, prm, dC, dF)
    got = {k: (None if v is None else v.cpu().numpy()) for k, v in g.items()}
    assert np.all(got["scales"][:, 2] == 0.0)
    got["scales2"] = got["scales"][:, :2]
    check_grads(got, ref, keys=("means", "scales2", "quats", "opacities", "sh"), tol=1e-3)
    check_grads(got, ref, keys=("features",), tol=1e-2)
    # the colour-only backward (no feature upstream) on the tensor-core kernel
    g0 = rast.backward(st, _t(dC), None)
    ref0 = surfel_ref_grads(sc, cams, prm, dC, None)
    got0 = {k: (None if v is None else v.cpu().numpy()) for k, v in g0.items()}
    got0["scales2"] = got0["scales"][:, :2]
    check_grads(got0, ref0, keys=("means", "scales2", "quats", "opacities", "sh"), tol=1e-3)
    # FHGS_PATH_TC gives the same forward
    rast.set_path(api.PATH_TC)
    rgb2, feat2 = rast.forward(st, feats)
    torch.cuda.synchronize()
    assert torch.equal(rgb2, rgb) and torch.equal(feat2, feat)
    rast.set_path(api.PATH_AUTO)
    with pytest.raises(api.FhgsError) as e:
        rast.fuse(t["means"], t["scales"], t["quats"], t["opacities"], t["sh"], cams[:1],
                  [torch.ones((48 * 40, 256), device=rgb.device)])
    assert e.value.status == api.ERR_UNSUPPORTED
    # FHGS_PATH_FP32 renders and differentiates the surfel scene on the CUDA cores (the FP32 bars)
    rast.set_path(api.PATH_FP32)
    rast.ctx.profile_read()
    rgb3, feat3 = rast.forward(st, feats)
    g3 = rast.backward(st, _t(dC), _t(dF))
    torch.cuda.synchronize()
    prof = rast.ctx.profile_read()
    assert "render_fwd_surfel" in prof and "render_bwd_surfel" in prof, prof
    check_surfel_image(dict(rgb=rgb3.cpu().numpy(), feat=feat3.cpu().numpy(), T=st["T"].cpu().numpy()), sc, cams,
                       prm)
    got3 = {k: (None if v is None else v.cpu().numpy()) for k, v in g3.items()}
    got3["scales2"] = got3["scales"][:, :2]
    check_grads(got3, ref, keys=("means", "scales2", "quats", "opacities", "sh", "features"), tol=1e-3)


def _surfel_ndfd_case(n, seed, D, cam, bf16):
    sc = surfel_scene(n, seed=seed, sh_degree=0, D=0)
    protos = synth.ndfd_prototypes(seed, D)
    f = synth.ndfd_features(seed, n, protos)
    fg = synth.ndfd_ground_truth(seed, 0, cam["height"], cam["width"], protos)
    if bf16:
        f, fg = synth.to_bf16(f), synth.to_bf16(fg)
    return sc, np.asarray(f, np.float64), np.asarray(fg, np.float64).reshape(-1, D)


@pytest.mark.parametrize("D,bf16", [(64, False), (256, True), (512, True)])
def test_surfel_ndfd_losses_and_gradients(D, bf16):
    """NDFD over surfel weights (Sec. 3.1-3.3; the paper's own combination):
    L_gt, L_cf and contributor counts against orc_ndfd_2dgs outside the
    surfel render's margin pixels, the gradients against orc_ndfd_2dgs_bwd
    within 1e-3 relative L2, SH and the third scale exactly zero."""
    cam = synth.look_at_camera(synth.ring_position(2.6, 35, 12), 64, 48)
    sc, f, fg = _surfel_ndfd_case(1200, 70 + D, D, cam, bf16)
    prm = dict(sh_degree=0)
    dt = torch.bfloat16 if bf16 else torch.float32
    rast = api.Rasterizer(0, sh_degree=0, geometry=api.GEOM_SURFEL)
    t = {k: _t(sc[k]) for k in ("means", "scales", "quats", "opacities", "sh")}
    feats, gt = _t(f, dt), _t(fg, dt)
    rast.ctx.profile(True)
    st = rast.prepare(t["means"], t["scales"], t["quats"], t["opacities"], t["sh"], [cam])
    nc = torch.empty(gt.shape[0], dtype=torch.int32, device=gt.device)
    Lgt, Lcf = rast.ndfd_forward(st, feats, gt, ncontrib=nc)
    P = cam["width"] * cam["height"]
    a, b = synth.upstream(17, P, 1)[0][:, 0].copy(), synth.upstream(18, P, 1)[0][:, 0].copy()
    g = rast.ndfd_backward(st, feats, gt, _t(a), _t(b))
    torch.cuda.synchronize()
    assert rast.ctx.sync_status() == api.OK
    prof = rast.ctx.profile_read()
    tc = bf16 and D == 512   # surfels take the tensor-core NDFD kernels at D = 512 (the 4-CTA layout)
    sfx = "_tc_surfel" if tc else "_surfel"
    assert "ndfd_fwd" + sfx in prof and "ndfd_bwd" + sfx in prof, prof
    if not tc:   # FHGS_PATH_TC is refused before any launch where the tensor-core kernels do not apply
        with pytest.raises(api.FhgsError) as e:
            rast.set_path(api.PATH_TC)
            rast.ndfd_forward(st, feats, gt)
        assert e.value.status == api.ERR_UNSUPPORTED
        rast.set_path(api.PATH_AUTO)
    ref = oracle.ndfd_2dgs(sc, cam, prm, f, fg)
    ok = oracle.surfel_forward(sc, cam, prm)["margin"].reshape(-1) > MARGIN_TOL
    check_margin_count(int((~ok).sum()), P, "surfel NDFD")
    for key, got in (("Lgt", Lgt), ("Lcf", Lcf)):
        err = np.abs(got.cpu().numpy() - ref[key].reshape(-1))[ok].max(initial=0)
        print(f"surfel NDFD D={D}: {key} err {err:.3g}")
        assert err <= 5e-5, (key, err)
    np.testing.assert_array_equal(nc.cpu().numpy()[ok], ref["ncontrib"].reshape(-1)[ok])
    assert (ref["ncontrib"] > 2).mean() > 0.1 and np.abs(ref["Lcf"]).max() > 1e-2
    gr = oracle.ndfd_2dgs_bwd(sc, cam, prm, f, fg, a, b)
    got = {k: v.cpu().numpy() for k, v in g.items()}
    assert np.all(got["scales"][:, 2] == 0.0) and np.all(got["sh"] == 0.0)
    got["scales2"] = got["scales"][:, :2]
    check_grads(got, gr, keys=("means", "scales2", "quats", "opacities"), tol=1e-3)
    if tc:  # the backward from the forward's saved end state gives the same gradients
        rast.ndfd_forward(st, feats, gt, save_state=True)
        g2 = rast.ndfd_backward(st, feats, gt, _t(a), _t(b))
        torch.cuda.synchronize()
        assert rast.ctx.sync_status() == api.OK
        for k in ("means", "scales", "quats", "opacities"):
            x, y = g2[k].cpu().numpy().astype(np.float64), got[k].astype(np.float64)
            assert np.linalg.norm(x - y) <= 1e-5 * np.linalg.norm(y), k
