"""Full-size workloads on the GPU, checked on sampled outputs.

* The 1M-Gaussian 1920x1080 D=512 BF16 view, in the launch configuration the
  benchmark times (tensor-core path, the library's own D split): bit-exact
  tile lists of the 64x64 crop at (928, 508), its image within the TC bars,
  and the gradients of an upstream gradient that is zero outside the crop
  (so the full-frame backward equals the oracle's crop backward).
* Sixteen cameras of uneven size (W in [640, 1600], H in [480, 900]) over
  500k Gaussians with D=256 BF16, rendered forward + backward in one launch
  per kernel, D split picked by the autotuner, the whole step captured in a
  CUDA graph and replayed: replays equal the eager step, and two cameras'
  centre crops (lists, image) and one crop's gradients match the oracle.

Bars as in test_gpu_tc: RGB 1e-5, `last` exact, features 1e-2 of max|F|,
footprint gradients 1e-3 and feature gradients 1e-2 relative L2.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2505_19154_gb300 import api, autotune, synth
from tests.test_gpu_parity import check_grads
from tests.helpers import MARGIN_TOL, check_margin_count

pytestmark = pytest.mark.gpu


def _dev():
    return torch.device("cuda", 0)


def _upload(scene, dev):
    t = {k: torch.from_numpy(np.ascontiguousarray(scene[k], np.float32)).to(dev)
         for k in ("means", "scales", "quats", "opacities", "sh")}
    t["features"] = torch.from_numpy(np.ascontiguousarray(scene["features"], np.float32)).to(dev).to(torch.bfloat16)
    return t


def _tile_rect(region):
    x0, y0, x1, y1 = region
    return (x0 // 16, y0 // 16, (x1 - 1) // 16, (y1 - 1) // 16)


def _cam_slices(cams):
    pix = np.cumsum([0] + [c["width"] * c["height"] for c in cams])
    tiles = np.cumsum([0] + [((c["width"] + 15) // 16) * ((c["height"] + 15) // 16) for c in cams])
    return pix, tiles


def compare_crop(rgb, feat, T, last, ranges, gids, cams, ci, region, scene, prm, D):
    """Tile lists of the crop's tiles and the crop's image of camera ci
    (device tensors over all cameras) against the oracle."""
    cam = cams[ci]
    pix, tiles = _cam_slices(cams)
    W = cam["width"]
    x0, y0, x1, y1 = region
    prep = oracle.prepare(scene, [cam], prm, tile_rect=_tile_rect(region))
    # lists: every tile of the crop, bit-exact
    tx0, ty0, tx1, ty1 = _tile_rect(region)
    tiles_x = (W + 15) // 16
    r_gpu = ranges[int(tiles[ci]):int(tiles[ci + 1])].cpu().numpy().astype(np.int64)
    r_ref = prep["lists"]["ranges"].astype(np.int64)
    g_ref = prep["lists"]["gids"]
    for ty in range(ty0, ty1 + 1):
        for tx in range(tx0, tx1 + 1):
            t = ty * tiles_x + tx
            a = gids[int(r_gpu[t, 0]):int(r_gpu[t, 1])].cpu().numpy().view(np.uint32)
            b = g_ref[int(r_ref[t, 0]):int(r_ref[t, 1])]
            np.testing.assert_array_equal(a, b, err_msg=f"camera {ci} tile {(tx, ty)}")
    # image of the crop
    rows = torch.arange(y0, y1, device=rgb.device)[:, None] * W + torch.arange(x0, x1, device=rgb.device)[None, :]
    idx = (rows.reshape(-1) + int(pix[ci])).long()
    ref = oracle.forward(scene, [cam], prm, scene["features"], region=region, prep=prep)[0]
    ok = ref["margin"].reshape(-1) > MARGIN_TOL
    check_margin_count(int((~ok).sum()), ok.size, f"camera {ci} crop")
    g_rgb = rgb[idx].cpu().numpy()
    assert np.abs(g_rgb - ref["rgb"].reshape(-1, 3))[ok].max(initial=0) <= 1e-5
    assert np.abs(T[idx].cpu().numpy() - ref["T"].reshape(-1))[ok].max(initial=0) <= 1e-5
    np.testing.assert_array_equal(last[idx].cpu().numpy()[ok], ref["last"].reshape(-1)[ok])
    fr = ref["feat"].reshape(-1, D)
    diff = np.abs(feat[idx].cpu().numpy() - fr)
    err = diff[ok].max(initial=0) / max(1.0, np.abs(fr).max())
    big = ok[:, None] & (np.abs(fr) >= 0.1 * np.abs(fr).max())
    rel = (diff[big] / np.abs(fr)[big]).max(initial=0)
    print(f"camera {ci} crop features: max abs err / max|F| {err:.3g}, "
          f"max rel err where |F| >= 0.1 max|F| {rel:.3g}")
    assert err <= 1e-2, err
    assert ref["ncontrib"].mean() > 10  # the crop is well inside the scene
    return prep, idx


def crop_upstream(cams, ci, region, D, seed, dev):
    """dL/drgb, dL/dfeat over all cameras: N(0,1) on camera ci's crop, 0 elsewhere."""
    pix, _ = _cam_slices(cams)
    P = int(pix[-1])
    x0, y0, x1, y1 = region
    dCc, dFc = synth.upstream(seed, (x1 - x0) * (y1 - y0), D)
    dC = torch.zeros((P, 3), device=dev)
    dF = torch.zeros((P, D), device=dev)
    W = cams[ci]["width"]
    rows = torch.arange(y0, y1, device=dev)[:, None] * W + torch.arange(x0, x1, device=dev)[None, :]
    idx = (rows.reshape(-1) + int(pix[ci])).long()
    dC[idx] = torch.from_numpy(np.asarray(dCc, np.float32)).to(dev)
    dF[idx] = torch.from_numpy(np.asarray(dFc, np.float32)).to(dev)
    return dC, dF, dCc, dFc


def _grads_np(g):
    return {k: (None if v is None else v.cpu().numpy()) for k, v in g.items()}


def test_config3_full_frame_in_bench_configuration():
    dev = _dev()
    scene, cams = synth.config3(0)
    D = 512
    prm = dict(sh_degree=3)
    t = _upload(scene, dev)
    rast = api.Rasterizer(0, sh_degree=3)  # automatic path and split, as the benchmark runs it
    rast.ctx.profile(True)
    st = rast.prepare(t["means"], t["scales"], t["quats"], t["opacities"], t["sh"], cams)
    rgb, feat = rast.forward(st, t["features"])
    dC, dF, dCc, dFc = crop_upstream(cams, 0, synth.CROP3, D, 3, dev)
    grads = rast.backward(st, dC, dF)
    torch.cuda.synchronize()
    assert rast.ctx.sync_status() == api.OK
    prof = rast.ctx.profile_read()
    assert "render_fwd_tc" in prof and "render_bwd_tc" in prof, prof
    prep, _ = compare_crop(rgb, feat, st["T"], st["last"], st["ranges"], st["gids"], cams, 0, synth.CROP3, scene,
                           prm, D)
    ref = oracle.backward(scene, cams, prm, scene["features"], [dCc], [dFc], region=synth.CROP3, prep=prep)
    g = _grads_np(grads)
    check_grads(g, ref, keys=("means", "scales", "quats", "opacities", "sh"), tol=1e-3)
    check_grads(g, ref, keys=("features",), tol=1e-2)


def _centre_crop(cam, size=64):
    x0 = (cam["width"] - size) // 2 // 16 * 16 + 5   # not tile-aligned: the crop spans 5 x 5 tiles
    y0 = (cam["height"] - size) // 2 // 16 * 16 + 3
    return (x0, y0, x0 + size, y0 + size)


def test_config4_sixteen_cameras_autotuned_graph():
    dev = _dev()
    scene, cams = synth.config4(0)
    assert len(cams) == 16
    assert len({(c["width"], c["height"]) for c in cams}) > 8
    D = 256
    prm = dict(sh_degree=3)
    t = _upload(scene, dev)
    a, b = 3, 11
    reg_a, reg_b = _centre_crop(cams[a]), _centre_crop(cams[b])
    dC, dF, dCc, dFc = crop_upstream(cams, a, reg_a, D, 4, dev)

    rast = api.Rasterizer(0, sh_degree=3, path=api.PATH_TC)
    st = rast.prepare(t["means"], t["scales"], t["quats"], t["opacities"], t["sh"], cams)
    rast.forward(st, t["features"])
    tuned = autotune.tune_splits(rast, st, t["features"], dC, dF, cams, use_cache=False)
    assert tuned["fwd"] in autotune.FWD_SPLITS and tuned["bwd"] in autotune.BWD_SPLITS
    assert len(tuned["times_ms"]) == sum(D % dn == 0 for dn in autotune.FWD_SPLITS + autotune.BWD_SPLITS)

    step = api.CapturedStep(rast, t["means"], t["scales"], t["quats"], t["opacities"], t["sh"], t["features"],
                            dC, dF, cams)
    o1 = step.replay()
    torch.cuda.synchronize()
    keep = {k: o1[k].clone() for k in ("rgb", "feat", "T", "last")}
    g1 = {k: v.clone() for k, v in o1["grads"].items()}
    o2 = step.replay()
    torch.cuda.synchronize()
    assert rast.ctx.sync_status() == api.OK
    # replays are the same computation: forward bit for bit, gradients up to
    # the order of the atomics
    for k in keep:
        assert torch.equal(keep[k], o2[k]), k
    for k, v in g1.items():
        if v is not None:
            assert torch.linalg.norm((v - o2["grads"][k]).double()) <= 1e-5 * torch.linalg.norm(v.double()), k
    # ... and the eager step with the same splits
    st_e = rast.prepare(t["means"], t["scales"], t["quats"], t["opacities"], t["sh"], cams)
    rgb_e, feat_e = rast.forward(st_e, t["features"])
    torch.cuda.synchronize()
    assert torch.equal(rgb_e, o2["rgb"]) and torch.equal(feat_e, o2["feat"])
    assert torch.equal(st_e["last"], o2["last"])

    n_inst = int(o2["count"].item())
    assert n_inst == st_e["n_instances"]
    for ci, reg in ((a, reg_a), (b, reg_b)):
        prep, _ = compare_crop(o2["rgb"], o2["feat"], o2["T"], o2["last"], o2["ranges"], o2["gids"], cams, ci,
                               reg, scene, prm, D)
        if ci == a:
            ref = oracle.backward(scene, [cams[a]], prm, scene["features"], [dCc], [dFc], region=reg, prep=prep)
            g = _grads_np(o2["grads"])
            check_grads(g, ref, keys=("means", "scales", "quats", "opacities", "sh"), tol=1e-3)
            check_grads(g, ref, keys=("features",), tol=1e-2)

    # the list cut inside the captured step (the bench's configuration): the
    # same forward bit for bit and the same gradients, from fewer instances
    rast_c = api.Rasterizer(0, sh_degree=3, path=api.PATH_TC, list_cut=1)
    rast_c.set_splits(tuned["fwd"], tuned["bwd"])
    step_c = api.CapturedStep(rast_c, t["means"], t["scales"], t["quats"], t["opacities"], t["sh"], t["features"],
                              dC, dF, cams)
    oc = step_c.replay()
    torch.cuda.synchronize()
    assert rast_c.ctx.sync_status() == api.OK
    for k in ("rgb", "feat", "T", "last"):
        assert torch.equal(oc[k], o2[k]), k
    for k, v in o2["grads"].items():
        if v is not None:
            assert torch.linalg.norm((v - oc["grads"][k]).double()) <= 1e-5 * torch.linalg.norm(v.double()), k
    assert int(oc["count"].item()) < n_inst
