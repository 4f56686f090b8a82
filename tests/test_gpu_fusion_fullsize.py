"""Feature fusion (Sec. 3.1) at the full size of the fusion workload: 3M
Gaussians, 1280x720 views, D=256 FP32 smooth feature maps.

* One full view against the oracle: every Gaussian's numerator and
  denominator, and the fused feature within 1e-4 relative where den > 1e-6.
  The oracle composites over the FP32 binning specification's footprints
  (the kernels' contribute/skip decisions rest on those); a Gaussian whose
  weights a near-threshold decision (within 1e-5) could move by more than
  the bar allows is checked against the bar plus that bound instead, and
  counted (at most 10 %; the bound is a worst case).
* All 64 views on the GPU with a constant map (the same unit vector at every
  pixel of every view): every Gaussian that some view sees must fuse to that
  constant, whatever its weights (the ratio of sums of w c over sums of w).
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2505_19154_gb300 import api, synth

pytestmark = pytest.mark.gpu


def _upload(scene, dev):
    return tuple(torch.from_numpy(np.ascontiguousarray(scene[k], np.float32)).to(dev)
                 for k in ("means", "scales", "quats", "opacities", "sh"))


def test_config5_one_full_view_against_oracle():
    dev = torch.device("cuda", 0)
    scene, views = synth.config5(0)
    view = views[0]
    D = 256
    fmap = synth.smooth_feature_map(0, 0, view["height"], view["width"], D)
    g = _upload(scene, dev)
    # decisions on the FP32 specification's footprints, as the kernels take them
    prep = oracle.prepare(scene, [view], dict(sh_degree=3), geometry="fp32")
    ref = oracle.fuse(scene, [view], [fmap], dict(sh_degree=3), prep=prep)
    for cut in (0, 1):  # full lists, then the rounds over depth segments
        rast = api.Rasterizer(0, sh_degree=3, list_cut=cut)
        out, num, den = rast.fuse(*g, [view], [torch.from_numpy(fmap.reshape(-1, D)).to(dev)])
        torch.cuda.synchronize()
        assert rast.ctx.sync_status() == api.OK
        _check_view(out, den, ref)


def _check_view(out, den, ref):
    den_g, den_r = den.cpu().numpy().astype(np.float64), ref["den"]
    seen = den_r > 1e-6
    assert seen.sum() > 2_000, seen.sum()  # the dense ball saturates within its outer shell
    assert np.abs(den_g - den_r).max() <= 1e-4 * max(1.0, den_r.max())
    # margin rule for fusion: where an oracle decision that settles a
    # contributor set lies within 1e-5 (relative) of its threshold, FP32 may
    # flip it.  wflip bounds the weight such flips could move; with unit-norm
    # maps the fused feature then moves by at most 2 wflip / den.  Gaussians
    # where that could exceed the bar are excluded and counted (at most 6 %
    # of the seen ones; 5.2 % in this view); every other seen Gaussian is held
    # to the plain 1e-4 bar.
    f_g = out.cpu().numpy().astype(np.float64)
    fn = np.maximum(np.linalg.norm(ref["out"], axis=1), 1e-30)
    risk = 2.0 * ref["wflip"] / np.maximum(den_r, 1e-30) / fn
    near = risk > 1e-4
    chk = seen & ~near
    rel = np.linalg.norm(f_g - ref["out"], axis=1) / fn
    stats = dict(seen=int(seen.sum()), near=int((seen & near).sum()), max_checked=float(rel[chk].max()),
                 p99_checked=float(np.percentile(rel[chk], 99)), max_near=float(rel[seen & near].max(initial=0)))
    print(stats)
    assert rel[chk].max() <= 1e-4, stats
    assert np.percentile(rel[chk], 99) <= 1e-5, stats
    # the excluded ones stay within the bar plus what their flips can explain
    assert np.all(rel[seen] <= 1e-4 + risk[seen]), stats
    assert (seen & near).sum() <= 0.06 * seen.sum(), stats
    assert np.all(out.cpu().numpy()[~seen & (den_r == 0)] == 0)


def test_config5_all_views_constant_map():
    dev = torch.device("cuda", 0)
    scene, views = synth.config5(0)
    assert len(views) == 64
    D = 256
    c = torch.from_numpy(synth.rng(7, 0).standard_normal(D).astype(np.float32))
    c /= torch.linalg.norm(c)
    P = views[0]["width"] * views[0]["height"]
    cmap = c.to(dev).expand(P, D).contiguous()   # 944 MB, shared by the 64 views
    g = _upload(scene, dev)
    rast = api.Rasterizer(0, sh_degree=3, list_cut=1)
    out, num, den = rast.fuse(*g, views, [cmap] * len(views))
    torch.cuda.synchronize()
    assert rast.ctx.sync_status() == api.OK
    seen = den > 1e-6
    assert int(seen.sum()) > 20_000  # 66k of the 3M Gaussians get weight in some view
    err = (out[seen] - c.to(dev)[None, :]).abs().max().item()
    assert err <= 1e-5, err
    assert torch.all(out[den == 0] == 0)
