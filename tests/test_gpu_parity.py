"""Parity of the CUDA path (through the C ABI) against the FP64 oracle.

Bars (stated per output):
  * tile keys, sorted Gaussian ids and tile ranges: bit-exact against the
    oracle's FP32 binning specification;
  * FP32 path: RGB and T_final within 1e-5 max abs, `last` exact, features
    within 1e-4 x max(1, max|F|) -- over pixels whose oracle decisions are
    not within 1e-5 (relative) of a threshold.  The feature bound follows
    from the arithmetic: w_i carries the FP32 product of up to ~200
    (1 - alpha) factors, a relative error eps of up to ~200 x 2^-24 x 2
    ~ 2.5e-5, so |dF| <= eps sum_i w_i |f_i| <= eps max|f| with sum w <= 1,
    and max|f| is a few times max|F| for N(0,1) features.  Margin pixels
    are counted and capped by tests.helpers.margin_cap (0.1 % of the pixels
    plus a few for small images); only decisions that settle the pixel's
    contributor set count;
  * gradients: ||g - g_ref||_2 / ||g_ref||_2 <= 1e-3 per parameter tensor;
  * fusion: per-Gaussian ||f - f_ref|| / ||f_ref|| <= 1e-4 where den > 1e-6.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2505_19154_gb300 import api, synth
from tests.helpers import MARGIN_TOL, axis_camera, check_margin_count, scene_from, small_random_scene

pytestmark = pytest.mark.gpu

if torch.cuda.is_available():
    DEV = torch.device("cuda", 0)


def _t(a, dtype=torch.float32):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).to(DEV).to(dtype)


def run_gpu(scene, cams, prm, path=api.PATH_FP32, feat_dtype=torch.float32, dC=None, dF=None, capacity=None):
    extra = {k: v for k, v in prm.items() if k not in ("sh_degree", "bg")}
    rast = api.Rasterizer(0, sh_degree=prm.get("sh_degree", 0), path=path, bg=prm.get("bg", (0.0, 0.0, 0.0)),
                          keep_keys=True, **extra)
    t = {k: _t(scene[k]) for k in ("means", "scales", "quats", "opacities", "sh")}
    feats = _t(scene["features"], feat_dtype) if scene.get("features") is not None else None
    st = rast.prepare(t["means"], t["scales"], t["quats"], t["opacities"], t["sh"], cams, capacity=capacity)
    rgb, feat = rast.forward(st, feats)
    out = dict(rgb=rgb.cpu().numpy(), feat=None if feat is None else feat.cpu().numpy(),
               T=st["T"].cpu().numpy(), last=st["last"].cpu().numpy(), count=st["n_instances"])
    n = out["count"]
    out["keys"] = st["keys"][:n].cpu().numpy().view(np.uint64)
    out["gids"] = st["gids"][:n].cpu().numpy().view(np.uint32)
    out["ranges"] = st["ranges"].cpu().numpy().view(np.uint32)
    if dC is not None:
        g = rast.backward(st, _t(dC), None if dF is None else _t(dF))
        out["grads"] = {k: (None if v is None else v.cpu().numpy()) for k, v in g.items()}
    torch.cuda.synchronize()
    assert rast.ctx.sync_status() == api.OK
    return out


def check_lists(out, prep):
    L = prep["lists"]
    assert out["count"] == len(L["keys"])
    np.testing.assert_array_equal(out["keys"], L["keys"])
    np.testing.assert_array_equal(out["gids"], L["gids"])
    np.testing.assert_array_equal(out["ranges"], L["ranges"])


def check_image(out, refs, cams, feat_tol=1e-4, rgb_tol=1e-5):
    off = 0
    n_margin = n_pix = 0
    for cam, ref in zip(cams, refs):
        P = cam["width"] * cam["height"]
        ok = ref["margin"].reshape(-1) > MARGIN_TOL
        n_margin += int((~ok).sum())
        n_pix += P
        rgb = out["rgb"][off:off + P]
        assert np.abs(rgb - ref["rgb"].reshape(-1, 3))[ok].max(initial=0) <= rgb_tol
        assert np.abs(out["T"][off:off + P] - ref["T"].reshape(-1))[ok].max(initial=0) <= 1e-5
        np.testing.assert_array_equal(out["last"][off:off + P][ok], ref["last"].reshape(-1)[ok])
        if ref["feat"] is not None and out["feat"] is not None:
            D = ref["feat"].shape[-1]
            fr = ref["feat"].reshape(-1, D)
            scale = max(1.0, np.abs(fr).max())
            diff = np.abs(out["feat"][off:off + P] - fr)
            err = diff[ok].max(initial=0) / scale
            # the stricter per-element relative error, on record (not asserted):
            # over the entries whose |F| is at least a tenth of max|F|
            big = ok[:, None] & (np.abs(fr) >= 0.1 * np.abs(fr).max())
            rel = (diff[big] / np.abs(fr)[big]).max(initial=0)
            print(f"features: max abs err / max|F| {err:.3g}, max rel err where |F| >= 0.1 max|F| {rel:.3g}")
            assert err <= feat_tol, err
        off += P
    check_margin_count(n_margin, n_pix, "image")
    return n_margin


def check_grads(got, ref, keys=("means", "scales", "quats", "opacities", "sh", "features"), tol=1e-3):
    for k in keys:
        if ref.get(k) is None:
            continue
        a, b = got[k].reshape(-1).astype(np.float64), ref[k].reshape(-1)
        nb = np.linalg.norm(b)
        rel = np.linalg.norm(a - b) / max(nb, 1e-30)
        assert rel <= tol, (k, rel, nb)


# ----------------------------------------------------------------- config 1
def test_config1_forward_lists_and_image():
    scene, cams = synth.config1(0)
    prm = dict(sh_degree=0)
    prep = oracle.prepare(scene, cams, prm)
    out = run_gpu(scene, cams, prm)
    check_lists(out, prep)
    refs = oracle.forward(scene, cams, prm, scene["features"], prep=prep)
    check_image(out, refs, cams)


def test_config1_backward():
    scene, cams = synth.config1(1)
    prm = dict(sh_degree=0, bg=(0.2, 0.3, 0.1))
    dC, dF = synth.upstream(1, 64 * 64, 16)
    prep = oracle.prepare(scene, cams, prm)
    out = run_gpu(scene, cams, prm, dC=dC, dF=dF)
    ref = oracle.backward(scene, cams, prm, scene["features"], [dC], [dF], prep=prep)
    check_grads(out["grads"], ref)


# ------------------------------------------------- ragged, multi-camera, SH3
def test_multicamera_ragged_sh3_forward_backward():
    sc = small_random_scene(3000, seed=21, sh_degree=3, D=24, spread=0.5)
    sc["features"] = sc["features"].astype(np.float32)
    cams = [synth.look_at_camera(synth.ring_position(3.0, a, e), w, h)
            for a, e, w, h in [(0, 0, 70, 50), (40, 20, 33, 47), (200, -25, 96, 64)]]
    prm = dict(sh_degree=3, bg=(0.1, 0.2, 0.3))
    sc32 = {k: (np.asarray(v, np.float32) if isinstance(v, np.ndarray) else v) for k, v in sc.items()}
    prep = oracle.prepare(sc32, cams, prm)
    P = [c["width"] * c["height"] for c in cams]
    dC, dF = synth.upstream(5, sum(P), 24)
    out = run_gpu(sc32, cams, prm, dC=dC, dF=dF)
    check_lists(out, prep)
    refs = oracle.forward(sc32, cams, prm, sc32["features"], prep=prep)
    check_image(out, refs, cams)
    offs = np.cumsum([0] + P)
    ref = oracle.backward(sc32, cams, prm, sc32["features"], [dC[offs[i]:offs[i + 1]] for i in range(3)],
                          [dF[offs[i]:offs[i + 1]] for i in range(3)], prep=prep)
    check_grads(out["grads"], ref)


def test_bf16_features_on_fp32_path():
    scene, cams = synth.config1(2)
    scene["features"] = synth.to_bf16(scene["features"])
    prm = dict(sh_degree=0)
    prep = oracle.prepare(scene, cams, prm)
    out = run_gpu(scene, cams, prm, feat_dtype=torch.bfloat16)
    refs = oracle.forward(scene, cams, prm, scene["features"], prep=prep)
    check_image(out, refs, cams)


# ----------------------------------------------------------------- config 2
@pytest.mark.slow
def test_config2_forward_backward():
    scene, cams = synth.config2(0)
    prm = dict(sh_degree=3)
    dC, dF = synth.upstream(2, 512 * 512, 128)
    prep = oracle.prepare(scene, cams, prm)
    out = run_gpu(scene, cams, prm, dC=dC, dF=dF)
    check_lists(out, prep)
    refs = oracle.forward(scene, cams, prm, scene["features"], prep=prep)
    check_image(out, refs, cams)
    ref = oracle.backward(scene, cams, prm, scene["features"], [dC], [dF], prep=prep)
    check_grads(out["grads"], ref)


# -------------------------------------------------------------- edge cases
def test_empty_and_all_culled_scenes():
    cam = axis_camera(W=40, H=24, fx=30.0)
    prm = dict(sh_degree=0, bg=(0.25, 0.5, 0.75))
    for sc in (scene_from(np.zeros((0, 3)), 0.1, feats=np.zeros((0, 8))),
               scene_from([[0, 0, -1.0], [0.1, 0, 0.1]], 0.1, feats=np.ones((2, 8)))):
        sc["opacities"] = np.asarray(sc["opacities"], np.float32)
        out = run_gpu(sc, [cam], prm, dC=np.ones((40 * 24, 3), np.float32), dF=np.ones((40 * 24, 8), np.float32))
        assert out["count"] == 0
        np.testing.assert_allclose(out["rgb"], np.tile([0.25, 0.5, 0.75], (40 * 24, 1)), atol=1e-7)
        assert (out["T"] == 1).all() and (out["last"] == 0).all() and (out["feat"] == 0).all()
        for k, v in out["grads"].items():
            assert v is None or not np.any(v), k


def test_near_degenerate_footprints_bit_exact_lists():
    """Needle-like Gaussians seen edge-on take the binary64 determinant path."""
    g = np.random.default_rng(3)
    n = 400
    means = g.normal(0, 0.3, (n, 3))
    scales = np.stack([np.full(n, 0.2), np.full(n, 1e-5), np.full(n, 1e-5)], 1)
    q = np.tile([1.0, 0, 0, 0], (n, 1)) + g.normal(0, 1e-3, (n, 4))
    sc = scene_from(means, scales, quats=q, opac=0.8, feats=g.normal(size=(n, 8)))
    sc = {k: (np.asarray(v, np.float32) if isinstance(v, np.ndarray) else v) for k, v in sc.items()}
    cam = axis_camera(W=80, H=64, fx=60.0, t=(0, 0, 2.5), cx=40.3, cy=31.7)
    cam["fx"] = cam["fy"] = 60.0
    prm = dict(sh_degree=0, dilation=0.0)
    prep = oracle.prepare(sc, [cam], prm)
    out = run_gpu(sc, [cam], prm)
    check_lists(out, prep)


def test_capacity_overflow_is_reported_not_faulted():
    scene, cams = synth.config1(0)
    rast = api.Rasterizer(0, sh_degree=0, path=api.PATH_FP32)
    t = {k: _t(scene[k]) for k in ("means", "scales", "quats", "opacities", "sh")}
    rast.capacity = 100
    st = rast.prepare(t["means"], t["scales"], t["quats"], t["opacities"], t["sh"], cams, check=False)
    assert int(st["count"].item()) > 100
    assert rast.ctx.sync_status() == api.ERR_CAPACITY
    assert rast.ctx.sync_status() == api.OK  # cleared


def test_non_finite_inputs_are_culled_and_reported():
    sc = small_random_scene(50, seed=4, sh_degree=0, D=8)
    sc = {k: (np.asarray(v, np.float32) if isinstance(v, np.ndarray) else v) for k, v in sc.items()}
    sc["means"][3, 0] = np.nan
    sc["scales"][7, 1] = np.inf
    cam = axis_camera(W=32, H=32, fx=30.0, t=(0, 0, 2.0))
    rast = api.Rasterizer(0, sh_degree=0, path=api.PATH_FP32, keep_keys=True)
    t = {k: _t(sc[k]) for k in ("means", "scales", "quats", "opacities", "sh")}
    st = rast.prepare(t["means"], t["scales"], t["quats"], t["opacities"], t["sh"], [cam], check=False)
    torch.cuda.synchronize()
    assert rast.ctx.sync_status() == api.ERR_NUMERIC
    gids = st["gids"][:int(st["count"].item())].cpu().numpy()
    assert 3 not in gids and 7 not in gids


def test_invalid_arguments_launch_nothing():
    scene, cams = synth.config1(0)
    rast = api.Rasterizer(0, sh_degree=0)
    t = {k: _t(scene[k]) for k in ("means", "scales", "quats", "opacities", "sh")}
    st = rast.prepare(t["means"], t["scales"], t["quats"], t["opacities"], t["sh"], cams)
    P = 64 * 64
    rgb = torch.empty((P, 3), device=DEV)
    T = torch.empty(P, device=DEV)
    last = torch.empty(P, dtype=torch.int32, device=DEV)
    f12 = torch.zeros((1024, 12), device=DEV)
    feat = torch.empty((P, 12), device=DEV)
    with pytest.raises(api.FhgsError) as e:
        rast.ctx.render_fwd(st["n"], st["proj"], st["bins"], f12, 12, st["cams"], rast.params, rgb, feat, T, last)
    assert e.value.status == api.ERR_UNSUPPORTED
    f16 = torch.zeros(1024 * 16 + 4, device=DEV)[1:].view(-1)[: 1024 * 16].view(1024, 16)
    feat16 = torch.empty((P, 16), device=DEV)
    with pytest.raises(api.FhgsError) as e:
        rast.ctx.render_fwd(st["n"], st["proj"], st["bins"], f16, 16, st["cams"], rast.params, rgb, feat16, T, last)
    assert e.value.status == api.ERR_ALIGNMENT
    bad = api.make_params(sh_degree=4)
    with pytest.raises(api.FhgsError) as e:
        rast.ctx.project(st["g"], st["cams"], bad, st["proj"])
    assert e.value.status == api.ERR_UNSUPPORTED


# ------------------------------------------------------------------ fusion
def test_fusion_matches_oracle_and_constant_map():
    sc = small_random_scene(2000, seed=31, sh_degree=0, D=0, spread=0.5)
    sc = {k: (np.asarray(v, np.float32) if isinstance(v, np.ndarray) else v) for k, v in sc.items()}
    views = [synth.look_at_camera(synth.ring_position(3.0, a, e), w, h)
             for a, e, w, h in [(0, 5, 72, 48), (60, -10, 64, 64), (150, 20, 50, 40)]]
    prm = dict(sh_degree=0)
    D = 16
    g = np.random.default_rng(0)
    maps = [g.normal(size=(v["height"], v["width"], D)).astype(np.float32) for v in views]
    ref = oracle.fuse(sc, views, maps, prm)
    rast = api.Rasterizer(0, sh_degree=0)
    t = {k: _t(sc[k]) for k in ("means", "scales", "quats", "opacities", "sh")}
    out, num, den = rast.fuse(t["means"], t["scales"], t["quats"], t["opacities"], t["sh"], views,
                              [_t(m).view(-1, D) for m in maps])
    out, den = out.cpu().numpy(), den.cpu().numpy()
    seen = ref["den"] > 1e-6
    assert seen.sum() > 200
    rel = np.linalg.norm(out[seen] - ref["out"][seen], axis=1) / np.linalg.norm(ref["out"][seen], axis=1)
    assert rel.max() <= 1e-4, rel.max()
    np.testing.assert_allclose(den, ref["den"], rtol=1e-4, atol=1e-6)
    assert (out[ref["den"] == 0] == 0).all()
    cmaps = [torch.full((v["height"] * v["width"], D), 0.7, device=DEV) for v in views]
    cout, _, _ = rast.fuse(t["means"], t["scales"], t["quats"], t["opacities"], t["sh"], views, cmaps)
    cout = cout.cpu().numpy()
    np.testing.assert_allclose(cout[seen], 0.7, rtol=1e-5)
