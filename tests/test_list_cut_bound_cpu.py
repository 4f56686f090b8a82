"""The geometry behind the list cut of binning (fhgs_params.list_cut = 1),
checked on the CPU against brute force.

The cut rests on two facts, both restated here from their definitions:
  * the box |dx| <= a, |dy| <= a sqrt(A/C) with 2 a^2 (A + |B| sqrt(A/C)) = q
    lies inside the ellipse A dx^2 + 2 B dx dy + C dy^2 <= q (its corners are
    the farthest points, and they are on the ellipse), so every pixel centre
    of a tile whose 16 x 16 centres fall in the box has q2 <= q and alpha >=
    min(alpha_max, op exp(-q/2));
  * a pixel that has not stopped after Gaussians with alpha_i >= a_i holds
    T = prod (1 - alpha_i) <= prod (1 - a_i) = exp(-sum -ln(1 - a_i)), so once
    that sum passes -ln(t_eps), T < t_eps and the pixel must have stopped.
The tile range follows the kernel's rule: tile k's centres are 16 k + 0.5 ..
16 k + 15.5, inside [m - h, m + h] for k in [ceil((m - h - 0.5) / 16),
floor((m + h - 15.5) / 16)].
"""
import math

import numpy as np


def box(A, B, C, q):
    rr = math.sqrt(A / C)
    a = math.sqrt(q / (2.0 * (A + abs(B) * rr)))
    return a, a * rr


def inner_tiles(m, h):
    return math.ceil((m - h - 0.5) / 16.0), math.floor((m + h - 15.5) / 16.0)


def q2(A, B, C, dx, dy):
    return A * dx * dx + 2.0 * B * dx * dy + C * dy * dy


def random_conic(g):
    # a screen covariance R diag(s1^2, s2^2) R^T + 0.3 I, inverted
    th = g.uniform(0.0, math.pi)
    s1, s2 = np.exp(g.uniform(0.0, 4.5, 2))
    c, s = math.cos(th), math.sin(th)
    S = np.array([[c, -s], [s, c]]) @ np.diag([s1 * s1, s2 * s2]) @ np.array([[c, s], [-s, c]]) + 0.3 * np.eye(2)
    K = np.linalg.inv(S)
    return K[0, 0], K[0, 1], K[1, 1]


def test_box_corners_lie_on_the_ellipse_and_the_box_inside():
    g = np.random.default_rng(11)
    for _ in range(2000):
        A, B, C = random_conic(g)
        q = g.choice([1.0, 3.0])
        a, b = box(A, B, C, q)
        # the corners attain the maximum of q2 over the box, and it is q
        corners = [q2(A, B, C, sx * a, sy * b) for sx in (-1, 1) for sy in (-1, 1)]
        assert abs(max(corners) - q) <= 1e-9 * q
        pts = g.uniform(-1.0, 1.0, (64, 2)) * np.array([a, b])
        assert (q2(A, B, C, pts[:, 0], pts[:, 1]) <= q * (1 + 1e-12)).all()


def test_inner_tile_centres_are_inside_the_shrunk_box():
    g = np.random.default_rng(12)
    hits = 0
    for _ in range(3000):
        A, B, C = random_conic(g)
        q = g.choice([1.0, 3.0])
        a0, b0 = box(A, B, C, q)
        ha, hb = a0 * (1 - 1e-3) - 1e-2, b0 * (1 - 1e-3) - 1e-2  # the kernel's margins
        if ha <= 0 or hb <= 0:
            continue
        mx, my = g.uniform(0.0, 1920.0), g.uniform(0.0, 1080.0)
        kx0, kx1 = inner_tiles(mx, ha)
        ky0, ky1 = inner_tiles(my, hb)
        for kx in range(kx0, kx1 + 1):
            for ky in range(ky0, ky1 + 1):
                hits += 1
                xs = 16 * kx + 0.5 + np.arange(16.0)
                ys = 16 * ky + 0.5 + np.arange(16.0)
                dx, dy = np.meshgrid(xs - mx, ys - my)
                assert (np.abs(dx) <= ha + 1e-9).all() and (np.abs(dy) <= hb + 1e-9).all()
                assert (q2(A, B, C, dx, dy) <= q * (1 - 1e-3)).all()
    assert hits > 100  # the sample covers tiles


def test_mass_bound_implies_stop():
    # prod (1 - a_i) < t_eps once sum -ln(1 - a_i) > -ln(t_eps); quantising
    # each term down (units of 1/256) keeps the bound conservative
    g = np.random.default_rng(13)
    t_eps = 1e-4
    thr = math.ceil(-math.log(t_eps) * 256) + 1
    for _ in range(500):
        a = g.uniform(1.0 / 255, 0.99, g.integers(1, 200))
        units = np.floor(-np.log1p(-a) * 256 * (1 - 1e-4)).astype(np.int64)
        if units.sum() >= thr:
            assert np.prod(1.0 - a) < t_eps
