"""NDFD at full size, in the launch configuration the bench times: 1M
Gaussians, one 1920x1080 view, D = 512 BF16 inputs from the device recipe.

The oracle cannot walk the whole frame, so the check samples the 64x64 crop at
(928, 508): L_gt, L_cf and the contributor counts of its 4,096 pixels against
the oracle over the crop's tile lists, and the gradients of upstream
gradients that are zero outside the crop.  With that upstream the full-frame
backward equals the oracle's crop backward: every Gaussian outside the crop's
lists must get exactly zero, every other one the oracle's gradient (same bars
as the small cases).
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2505_19154_gb300 import api, synth
from tests.test_gpu_ndfd import L_TOL
from tests.test_gpu_parity import check_grads
from tests.helpers import MARGIN_TOL, check_margin_count

pytestmark = pytest.mark.gpu


def test_ndfd_fullsize_crop():
    dev = torch.device("cuda", 0)
    N, D = 1_000_000, 512
    scene, cams = synth.config3(0, n=N, D=0)
    cam = cams[0]
    W = cam["width"]
    prm = dict(sh_degree=3)
    feats, fgt = synth.ndfd_inputs_device(0, N, cams, D, dev)
    x0, y0, x1, y1 = synth.CROP3
    pix = torch.tensor([y * W + x for y in range(y0, y1) for x in range(x0, x1)], device=dev)
    g = synth.rng(11, 5)
    a = torch.zeros(fgt.shape[0], device=dev)
    b = torch.zeros(fgt.shape[0], device=dev)
    a_c = g.standard_normal(pix.numel()).astype(np.float32)
    b_c = g.standard_normal(pix.numel()).astype(np.float32)
    a[pix] = torch.from_numpy(a_c).to(dev)
    b[pix] = torch.from_numpy(b_c).to(dev)

    rast = api.Rasterizer(0, sh_degree=3)
    t = [torch.from_numpy(np.ascontiguousarray(scene[k], np.float32)).to(dev)
         for k in ("means", "scales", "quats", "opacities", "sh")]
    st = rast.prepare(*t, cams)
    nc = torch.empty(fgt.shape[0], dtype=torch.int32, device=dev)
    Lgt, Lcf = rast.ndfd_forward(st, feats, fgt, ncontrib=nc)
    gr = rast.ndfd_backward(st, feats, fgt, a, b)
    torch.cuda.synchronize()
    assert rast.ctx.sync_status() == api.OK
    got = dict(Lgt=Lgt[pix].cpu().numpy(), Lcf=Lcf[pix].cpu().numpy(), nc=nc[pix].cpu().numpy())
    grads = {k: v.cpu().numpy() for k, v in gr.items()}

    # the oracle over the crop's tiles; its lists hold the Gaussians renumbered 0..U-1
    prep = oracle.prepare(scene, cams, prm, tile_rect=(x0 // 16, y0 // 16, (x1 - 1) // 16, (y1 - 1) // 16))
    uniq, inv = np.unique(prep["lists"]["gids"], return_inverse=True)
    lists = inv.astype(np.uint32)
    ranges = np.ascontiguousarray(prep["lists"]["ranges"])
    rec = prep["recs"][0][uniq]
    fc = feats[torch.from_numpy(uniq.astype(np.int64)).to(dev)].float().cpu().numpy()
    fg = fgt[pix].float().cpu().numpy()
    ref = oracle.ndfd(rec, fc, lists, ranges, cam, prm, fg, region=synth.CROP3)
    margin = oracle.render(rec, None, lists, ranges, cam, prm, region=synth.CROP3)["margin"].reshape(-1)
    ok = margin > MARGIN_TOL
    check_margin_count(int((~ok).sum()), ok.size, "NDFD crop")
    for k in ("Lgt", "Lcf"):
        err = np.abs(got[k] - ref[k].reshape(-1))[ok].max()
        assert err <= L_TOL, (k, err)
    np.testing.assert_array_equal(got["nc"][ok], ref["ncontrib"].reshape(-1)[ok])
    assert ref["Lcf"].max() > 1e-2 and ref["ncontrib"].mean() > 10

    g2 = oracle.ndfd_bwd(rec, fc, lists, ranges, cam, prm, synth.CROP3, fg, a_c, b_c)
    sub = {k: np.asarray(scene[k])[uniq] for k in ("means", "scales", "quats", "opacities", "sh")}
    sub["sh_degree"] = 3
    gp = oracle.project_bwd(sub, cam, prm, rec, g2)
    ref_g = dict(means=gp["means"], scales=gp["scales"], quats=gp["quats"], opacities=g2["op"])
    check_grads({k: grads[k][uniq] for k in ref_g}, ref_g, keys=tuple(ref_g), tol=1e-3)
    outside = np.ones(N, bool)
    outside[uniq] = False
    for k in ("means", "scales", "quats", "opacities", "sh"):
        assert not np.any(grads[k][outside]), k
    assert not np.any(grads["sh"])
