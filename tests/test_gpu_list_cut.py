"""The list cut of fhgs_bin_sort (params.list_cut = 1) against the full lists.

The cut drops, per tile, the entries after the depth segment by whose end an
opacity bound proves that every pixel of the tile has stopped compositing.
What must hold, and is checked here on scenes dense enough to saturate:
  * each cut list is a prefix of the tile's full list (bit-exact ids), and the
    instance count is the sum of the cut lengths;
  * the forward outputs (RGB, features, T_final, last) over the cut lists are
    bit-identical to those over the full lists, on the FP32 and tensor-core
    paths; the gradients agree to the order of their float atomics (1e-4
    relative L2: sums with cancellation move by a few 1e-6 between two runs
    on the same lists);
  * the NDFD losses and gradients agree the same way, and so do the fused
    features (fusion bins each view with the same cut);
  * where the cut does not apply (2DGS surfels, a camera grid too large for
    the count pass) the lists stay full.
"""
import numpy as np
import pytest
import torch

from paper_2505_19154_gb300 import api, synth

pytestmark = pytest.mark.gpu

if torch.cuda.is_available():
    DEV = torch.device("cuda", 0)


def _t(a, dtype=torch.float32):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).to(DEV).to(dtype)


def _inputs(scene, feat_dtype=torch.float32):
    t = {k: _t(scene[k]) for k in ("means", "scales", "quats", "opacities", "sh")}
    feats = _t(scene["features"], feat_dtype) if scene.get("features") is not None else None
    return t, feats


def _lists(st):
    n = st["n_instances"]
    gids = st["gids"][:n].cpu().numpy().view(np.uint32)
    ranges = st["ranges"].cpu().numpy().view(np.uint32)
    return gids, ranges


def _prepare(scene, cams, cut, path=api.PATH_FP32, geometry=0, **kw):
    rast = api.Rasterizer(0, sh_degree=scene["sh_degree"], path=path, list_cut=cut, geometry=geometry, **kw)
    t, _ = _inputs(scene)
    st = rast.prepare(t["means"], t["scales"], t["quats"], t["opacities"], t["sh"], cams)
    st["inputs"] = t  # the state holds raw pointers to these tensors: keep them alive
    return rast, st


def check_prefix(full, cut):
    """Every cut list is a prefix of the full list of its tile."""
    gf, rf = full
    gc, rc = cut
    lf = rf[:, 1].astype(np.int64) - rf[:, 0]
    lc = rc[:, 1].astype(np.int64) - rc[:, 0]
    assert (lc <= lf).all()
    assert int(lc.sum()) == len(gc)
    for t in np.nonzero(lc)[0]:
        np.testing.assert_array_equal(gc[rc[t, 0]:rc[t, 1]], gf[rf[t, 0]:rf[t, 0] + lc[t]])
    return int(lc.sum()), int(lf.sum())


def _rel(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30))


def _render(scene, cams, cut, path, feat_dtype, dC, dF):
    rast, st = _prepare(scene, cams, cut, path=path)
    _, feats = _inputs(scene, feat_dtype)
    rgb, feat = rast.forward(st, feats)
    g = rast.backward(st, _t(dC), _t(dF))
    torch.cuda.synchronize()
    assert rast.ctx.sync_status() == api.OK
    out = dict(rgb=rgb.cpu().numpy(), feat=feat.cpu().numpy(), T=st["T"].cpu().numpy(),
               last=st["last"].cpu().numpy(), lists=_lists(st),
               grads={k: v.cpu().numpy() for k, v in g.items() if v is not None})
    return out


@pytest.mark.parametrize("grow", [1.0, 4.0])
@pytest.mark.parametrize("path,feat_dtype", [(api.PATH_FP32, torch.float32), (api.PATH_TC, torch.bfloat16)])
def test_cut_lists_render_like_full_lists(path, feat_dtype, grow):
    # config-2 distributions (100k Gaussians, SH3) on a 512x512 view and two
    # ragged cameras; with the scales grown 4x, Gaussians cover whole tiles and
    # the bound closes most tiles of the dense ball early
    scene = synth.make_scene(100_000, 3, "normal", sh_degree=3, D=128)
    scene["scales"] = (scene["scales"] * grow).astype(np.float32)
    if feat_dtype == torch.bfloat16:
        scene["features"] = synth.to_bf16(scene["features"])
    cams = [synth.look_at_camera([0.0, 0.0, -4.0], 512, 512),
            synth.look_at_camera(synth.ring_position(4.0, 70.0, 20.0), 333, 217),
            synth.look_at_camera(synth.ring_position(4.0, 200.0, -10.0), 250, 401)]
    P = sum(c["width"] * c["height"] for c in cams)
    dC, dF = synth.upstream(5, P, 128)
    full = _render(scene, cams, 0, path, feat_dtype, dC, dF)
    cut = _render(scene, cams, 1, path, feat_dtype, dC, dF)
    n_cut, n_full = check_prefix(full["lists"], cut["lists"])
    print(f"instances: cut {n_cut}, full {n_full}")
    if grow > 1.0:
        assert n_cut < 0.5 * n_full, (n_cut, n_full)
    for k in ("rgb", "feat", "T", "last"):
        np.testing.assert_array_equal(cut[k], full[k], err_msg=k)
    for k, v in full["grads"].items():
        assert _rel(cut["grads"][k], v) <= 1e-4, k


def test_cut_lists_ndfd_like_full_lists():
    D = 256
    scene = synth.make_scene(60_000, 4, "normal", sh_degree=0, D=D)
    scene["features"] = synth.to_bf16(scene["features"] / np.linalg.norm(scene["features"], axis=1, keepdims=True))
    cams = [synth.look_at_camera([0.0, 0.0, -4.0], 320, 240)]
    P = 320 * 240
    gt = synth.rng(9, 0).standard_normal((P, D)).astype(np.float32)
    gt /= np.linalg.norm(gt, axis=1, keepdims=True)
    res = []
    for cut in (0, 1):
        rast, st = _prepare(scene, cams, cut, path=api.PATH_AUTO)
        _, feats = _inputs(scene, torch.bfloat16)
        fgt = _t(gt, torch.bfloat16)
        Lgt, Lcf = rast.ndfd_forward(st, feats, fgt)
        g = rast.ndfd_backward(st, feats, fgt, torch.ones_like(Lgt), torch.full_like(Lcf, 0.5))
        torch.cuda.synchronize()
        assert rast.ctx.sync_status() == api.OK
        res.append((Lgt.cpu().numpy(), Lcf.cpu().numpy(),
                    {k: v.cpu().numpy() for k, v in g.items() if v is not None}, _lists(st)))
    check_prefix(res[0][3], res[1][3])
    np.testing.assert_array_equal(res[1][0], res[0][0])
    np.testing.assert_array_equal(res[1][1], res[0][1])
    for k, v in res[0][2].items():
        assert _rel(res[1][2][k], v) <= 1e-4, k


def test_cut_lists_fuse_like_full_lists():
    D = 64
    scene = synth.make_scene(80_000, 6, "normal", sh_degree=0)
    views = [synth.look_at_camera(synth.ring_position(4.0, a, 10.0), 300, 200) for a in (0.0, 120.0)]
    maps = [_t(synth.smooth_feature_map(7, v, 200, 300, D)) for v in range(len(views))]
    t, _ = _inputs(scene)
    outs = []
    for cut in (0, 1):
        rast = api.Rasterizer(0, sh_degree=0, path=api.PATH_AUTO, list_cut=cut)
        f, num, den = rast.fuse(t["means"], t["scales"], t["quats"], t["opacities"], t["sh"], views, maps)
        torch.cuda.synchronize()
        assert rast.ctx.sync_status() == api.OK
        outs.append((f.cpu().numpy(), den.cpu().numpy()))
    assert _rel(outs[1][1], outs[0][1]) <= 1e-5
    assert _rel(outs[1][0], outs[0][0]) <= 1e-5


def test_cut_not_applied_to_surfels_or_large_grids():
    scene = synth.make_scene(20_000, 8, "normal", sh_degree=0)
    cams = [synth.look_at_camera([0.0, 0.0, -4.0], 256, 256)]
    _, full = _prepare(scene, cams, 0, geometry=api.GEOM_SURFEL)
    _, cut = _prepare(scene, cams, 1, geometry=api.GEOM_SURFEL)
    for a, b in zip(_lists(full), _lists(cut)):
        np.testing.assert_array_equal(a, b)
    # 3840x2160: (241 x 136) cells, two difference arrays do not fit
    big = [synth.look_at_camera([0.0, 0.0, -4.0], 3840, 2160)]
    _, full = _prepare(scene, big, 0)
    _, cut = _prepare(scene, big, 1)
    for a, b in zip(_lists(full), _lists(cut)):
        np.testing.assert_array_equal(a, b)


def test_cut_empty_scene():
    scene = synth.make_scene(1000, 9, "normal", sh_degree=0)
    scene["means"][:, 2] = -10.0  # all behind the camera
    cams = [synth.look_at_camera([0.0, 0.0, -4.0], 64, 64)]
    rast, st = _prepare(scene, cams, 1)
    assert st["n_instances"] == 0
    assert rast.ctx.sync_status() == api.OK
