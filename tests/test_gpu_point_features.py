"""Parity of the point-to-feature assignment (the CUDA path through the C
ABI) against the oracle.  The view and pixel are integer decisions of a
binary32 projection that both sides specify operation by operation, and the
feature is a copy: all three must match bit for bit.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2505_19154_gb300 import api, synth

pytestmark = pytest.mark.gpu


def run_case(pts, views, maps, u):
    dev = torch.device("cuda", 0)
    ctx = api.Context(0)
    params = api.make_params()
    tmaps = [torch.from_numpy(np.ascontiguousarray(m.reshape(-1, m.shape[-1]), np.float32)).to(dev) for m in maps]
    out, view, pixel = api.point_features(ctx, torch.from_numpy(np.asarray(pts, np.float32)).to(dev), views, tmaps,
                                          torch.from_numpy(np.asarray(u, np.float32)).to(dev), params)
    torch.cuda.synchronize()
    assert ctx.sync_status() == api.OK
    prof_ok = api.Context.launch_count() > 0
    ref = oracle.point_features(pts, views, [m.astype(np.float32) for m in maps], u)
    got_v, got_p = view.cpu().numpy(), pixel.cpu().numpy()
    np.testing.assert_array_equal(got_v, ref["view"])
    np.testing.assert_array_equal(got_p, ref["pixel"])
    np.testing.assert_array_equal(out.cpu().numpy(), ref["features"].astype(np.float32))
    assert prof_ok
    return ref


@pytest.mark.parametrize("n_views,D", [(6, 64), (70, 8)])
def test_point_features_match_oracle(n_views, D):
    g = synth.rng(21, n_views)
    views = [synth.look_at_camera(synth.ring_position(3.0, 360.0 * v / n_views, 25.0 * np.sin(v)),
                                  int(g.integers(40, 97)), int(g.integers(30, 71))) for v in range(n_views)]
    pts = g.uniform(-1.3, 1.3, (20011, 3)).astype(np.float32)
    pts[:7] = [0, 60, 0]           # seen by no view
    maps = [g.standard_normal((v["height"], v["width"], D)).astype(np.float32) for v in views]
    u = g.uniform(0, 1, len(pts)).astype(np.float32)
    ref = run_case(pts, views, maps, u)
    assert (ref["view"] >= 0).mean() > 0.5 and (ref["count"] > 1).mean() > 0.3 and (ref["view"][:7] == -1).all()


def test_point_features_bad_arguments():
    ctx = api.Context(0)
    params = api.make_params()
    dev = torch.device("cuda", 0)
    views = [synth.look_at_camera(synth.ring_position(3.0, 0, 0), 32, 24)]
    m = torch.zeros((32 * 24, 12), device=dev)
    with pytest.raises(api.FhgsError) as e:
        api.point_features(ctx, torch.zeros((4, 3), device=dev), views, [m], torch.zeros(4, device=dev), params)
    assert e.value.status == api.ERR_UNSUPPORTED   # D = 12 is not a multiple of 8
    big = torch.zeros(32 * 24 * 16 + 4, device=dev)
    with pytest.raises(api.FhgsError) as e:
        api.point_features(ctx, torch.zeros((4, 3), device=dev), views, [big[1:1 + 32 * 24 * 16].view(-1, 16)],
                           torch.zeros(4, device=dev), params)
    assert e.value.status == api.ERR_ALIGNMENT
