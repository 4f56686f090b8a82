"""Pins of the oracle's point-to-feature assignment (Sec. 3.1; App. A,
"PointsFeatureFusion"), no GPU.

(a) a point on a camera's optical axis lands on the pixel holding the
    principal point, and is culled in front of the near plane;
(b) the visible-view count equals an FP64 projection count for points away
    from the image edges;
(c) the draw: u = 0 takes the first visible view, u -> 1 the last, and
    u = (k + 1/2)/|M| the k-th, in view order;
(d) the chosen pixel equals the FP64 projection's floor away from pixel
    boundaries, and the feature is that pixel's map entry exactly;
(e) a point no view sees gets view -1 and zeros.
"""
import numpy as np

import oracle
from paper_2505_19154_gb300 import synth
from tests.helpers import axis_camera


def _views(n=6, W=80, H=60):
    return [synth.look_at_camera(synth.ring_position(3.0, 360.0 * v / n, 10.0 * (v % 3 - 1)), W, H)
            for v in range(n)]


def _proj64(means, cam):
    w2c = np.asarray(cam["w2c"], np.float64).reshape(3, 4)
    c = means @ w2c[:, :3].T + w2c[:, 3]
    x = cam["fx"] * c[:, 0] / c[:, 2] + cam["cx"]
    y = cam["fy"] * c[:, 1] / c[:, 2] + cam["cy"]
    return x, y, c[:, 2]


def test_point_on_the_axis_lands_on_the_principal_point():
    cam = axis_camera(W=64, H=40, fx=50.0, cx=20.25, cy=30.75)
    maps = [np.arange(64 * 40 * 2, dtype=np.float64).reshape(40, 64, 2)]
    r = oracle.point_features([[0.0, 0.0, 3.0]], [cam], maps, [0.3])
    assert r["view"][0] == 0 and r["count"][0] == 1
    assert r["pixel"][0] == 30 * 64 + 20
    np.testing.assert_array_equal(r["features"][0], maps[0][30, 20])
    # the near plane: depth 0.1 is culled (z <= znear = 0.2), 0.25 is seen
    r = oracle.point_features([[0.0, 0.0, 0.1], [0.0, 0.0, 0.25]], [cam], maps, [0.3, 0.3])
    assert list(r["view"]) == [-1, 0]


def test_counts_and_pixels_match_fp64_projection_away_from_edges():
    views = _views()
    g = synth.rng(3, 9)
    pts = g.uniform(-1.2, 1.2, (4000, 3))
    D = 3
    maps = [g.standard_normal((v["height"], v["width"], D)) for v in views]
    u = g.uniform(0, 1, 4000).astype(np.float32)
    r = oracle.point_features(pts, views, maps, u)
    vis = []
    near = np.zeros(len(pts), bool)
    for v in views:
        x, y, z = _proj64(pts, v)
        ok = (z > 0.2) & (x >= 0) & (x < v["width"]) & (y >= 0) & (y < v["height"])
        # within 1e-3 px of an edge, of a pixel boundary, or of the near plane the FP32 decision may differ
        fx, fy = x - np.floor(x), y - np.floor(y)
        near |= (np.minimum(fx, 1 - fx) < 1e-3) | (np.minimum(fy, 1 - fy) < 1e-3) | (np.abs(z - 0.2) < 1e-4)
        vis.append((ok, x, y))
    count = np.sum([ok for ok, _, _ in vis], axis=0)
    far = ~near
    assert far.mean() > 0.95
    np.testing.assert_array_equal(r["count"][far], count[far])
    checked = 0
    for i in np.nonzero(far & (count > 0))[0]:
        seen = [v for v in range(len(views)) if vis[v][0][i]]
        k = min(int(np.float32(u[i]) * np.float32(len(seen))), len(seen) - 1)
        v = seen[k]
        assert r["view"][i] == v
        x, y = vis[v][1][i], vis[v][2][i]
        assert r["pixel"][i] == int(np.floor(y)) * views[v]["width"] + int(np.floor(x))
        np.testing.assert_array_equal(r["features"][i], maps[v][int(np.floor(y)), int(np.floor(x))])
        checked += 1
    assert checked > 2000 and (count > 1).mean() > 0.5


def test_the_draw_walks_the_visible_views_in_order():
    views = _views(4)
    pt = np.zeros((1, 3))          # the ring's centre: every view sees it
    maps = [np.full((v["height"], v["width"], 1), float(i)) for i, v in enumerate(views)]
    for k in range(4):
        r = oracle.point_features(pt, views, maps, [(k + 0.5) / 4])
        assert r["count"][0] == 4 and r["view"][0] == k and r["features"][0, 0] == k
    assert oracle.point_features(pt, views, maps, [0.0])["view"][0] == 0
    assert oracle.point_features(pt, views, maps, [np.nextafter(np.float32(1), np.float32(0))])["view"][0] == 3


def test_unseen_point_gets_nothing():
    views = _views(3)
    maps = [np.ones((v["height"], v["width"], 4)) for v in views]
    r = oracle.point_features([[0.0, 50.0, 0.0], [0.0, -50.0, 0.0]], views, maps, [0.5, 0.5])   # straight above and below the ring
    assert (r["view"] == -1).all() and (r["count"] == 0).all() and not r["features"].any()
