"""Small scene/camera builders shared by the tests (no splatting arithmetic)."""
import numpy as np

from paper_2505_19154_gb300 import synth


def axis_camera(W=64, H=64, fx=50.0, fy=None, cx=None, cy=None, t=(0.0, 0.0, 0.0)):
    """Camera at the world origin (identity rotation) or translated by t."""
    w2c = np.zeros((3, 4))
    w2c[:3, :3] = np.eye(3)
    w2c[:, 3] = t
    return dict(width=W, height=H, fx=fx, fy=fx if fy is None else fy,
                cx=W / 2.0 if cx is None else cx, cy=H / 2.0 if cy is None else cy, w2c=w2c)


def scene_from(means, scales, quats=None, opac=None, colors=None, sh=None, feats=None):
    means = np.atleast_2d(np.asarray(means, np.float64))
    n = len(means)
    scales = np.broadcast_to(np.asarray(scales, np.float64), (n, 3)).copy()
    quats = (np.tile([1.0, 0, 0, 0], (n, 1)) if quats is None
             else np.atleast_2d(np.asarray(quats, np.float64)))
    opac = np.full(n, 0.5) if opac is None else np.broadcast_to(np.asarray(opac, np.float64), (n,)).copy()
    if sh is None:
        colors = np.full((n, 3), 0.5) if colors is None else np.atleast_2d(np.asarray(colors, np.float64))
        # degree-0 coefficient giving exactly `colors`: c = C0 * sh0 + 0.5
        sh = ((colors - 0.5) * (2.0 * np.sqrt(np.pi)))[:, None, :]
    s = dict(means=means, scales=scales, quats=quats, opacities=opac, sh=np.asarray(sh, np.float64),
             sh_degree=int(round(np.sqrt(np.asarray(sh).shape[1]))) - 1)
    if feats is not None:
        s["features"] = np.atleast_2d(np.asarray(feats, np.float64))
    return s


def small_random_scene(n=40, seed=0, sh_degree=3, D=8, spread=0.5):
    g = synth.rng(seed, 77)
    means = g.normal(0.0, spread, (n, 3))
    scales = np.exp(g.uniform(-3.0, -1.8, (n, 3)))
    q = g.normal(0.0, 1.0, (n, 4))
    opac = 1.0 / (1.0 + np.exp(-g.normal(0.0, 1.0, n)))
    K = (sh_degree + 1) ** 2
    sh = g.normal(0.0, 0.3, (n, K, 3))
    sh[:, 0, :] += 0.5
    feats = g.normal(0.0, 1.0, (n, D)) if D else None
    s = dict(means=means, scales=scales, quats=q, opacities=opac, sh=sh, sh_degree=sh_degree)
    if D:
        s["features"] = feats
    return s


# Margin rule for image comparisons (GPU FP32 against the FP64 oracle).  A
# pixel is excluded from the element-wise bars when one of the decisions that
# settle its contributor set (the ellipse cutoff of a Gaussian that would pass
# the alpha test there, the alpha_min test, the stop rule) lies within
# MARGIN_TOL (relative) of its threshold in the oracle: the largest FP32
# error of q^2 measured near the cutoff is 2.7e-6 relative, so such a
# decision may come out the other way in FP32.  The excluded pixels are
# counted; at most 0.1 % of the compared pixels plus MARGIN_SLACK pixels (one
# ellipse edge's worth, for images of a few thousand pixels) may be excluded.
MARGIN_TOL = 1e-5
MARGIN_SLACK = 8


def margin_cap(n_pix: int) -> float:
    return 1e-3 * n_pix + MARGIN_SLACK


def check_margin_count(n_margin: int, n_pix: int, what: str = "") -> None:
    print(f"margin pixels {what}: {n_margin} of {n_pix} ({100.0 * n_margin / max(n_pix, 1):.3f} %)")
    assert n_margin <= margin_cap(n_pix), (what, n_margin, n_pix)
