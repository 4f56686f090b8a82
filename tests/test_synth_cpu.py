"""The seeded input recipes (the paper's datasets stand in as synthetic
scenes): reproducible, with the stated distributions and shapes."""
import numpy as np

from paper_2505_19154_gb300 import synth


def test_philox_streams_are_reproducible_and_distinct():
    a = synth.rng(3, 7).standard_normal(1000)
    b = synth.rng(3, 7).standard_normal(1000)
    c = synth.rng(3, 8).standard_normal(1000)
    np.testing.assert_array_equal(a, b)
    assert np.abs(a - c).max() > 0.1


def test_scene_distributions():
    sc = synth.make_scene(20000, 0, "normal", sh_degree=3, D=8, feat_dtype="bf16")
    assert sc["means"].shape == (20000, 3) and np.abs(sc["means"]).max() <= 2.0
    assert abs(sc["means"].std() - 0.6) < 0.03
    ls = np.log(sc["scales"])
    assert ls.min() >= -5.0 - 1e-6 and ls.max() <= -2.0 + 1e-6
    np.testing.assert_allclose(np.linalg.norm(sc["quats"], axis=1), 1.0, atol=1e-6)
    assert sc["sh"].shape == (20000, 16, 3) and abs(sc["sh"].std() - 0.2) < 0.01
    assert 0.0 < sc["opacities"].min() and sc["opacities"].max() < 1.0
    f = sc["features"]
    np.testing.assert_array_equal(f, synth.to_bf16(f))  # BF16-representable


def test_config4_cameras_follow_the_recipe():
    cams = synth.config4_cameras(0)
    assert len(cams) == 16
    for i, c in enumerate(cams):
        assert 640 <= c["width"] <= 1600 and 480 <= c["height"] <= 900
        R, t = np.asarray(c["w2c"])[:, :3], np.asarray(c["w2c"])[:, 3]
        centre = -R.T @ t
        assert abs(np.linalg.norm(centre) - 4.0) < 1e-9
        el = np.degrees(np.arcsin(-centre[1] / 4.0))
        assert -30.0 <= el <= 30.0
        # looks at the origin: the optical axis passes through it
        np.testing.assert_allclose((R @ np.zeros(3) + t)[:2], 0.0, atol=1e-9)


def test_smooth_feature_map_is_normalised_and_smooth():
    m = synth.smooth_feature_map(0, 0, 48, 64, 16)
    assert m.shape == (48, 64, 16) and m.dtype == np.float32
    np.testing.assert_allclose(np.linalg.norm(m, axis=-1), 1.0, atol=1e-5)
    # sigma = 8 px: neighbouring pixels are strongly correlated, distant ones not
    near = np.mean(np.sum(m[:, 1:] * m[:, :-1], axis=-1))
    far = np.mean(np.abs(np.sum(m[:, 40:] * m[:, :-40], axis=-1)))
    assert near > 0.95 and far < 0.5


def test_ndfd_recipes_follow_their_description():
    """Unit features clustered around unit prototypes (cosine to the own
    prototype from about 0.98 down to about 0.3), a ground-truth map of
    constant-label blocks, and the device recipe (run here on the CPU) with
    the same structure."""
    import torch
    D = 256
    P = synth.ndfd_prototypes(3, D)
    np.testing.assert_allclose(np.linalg.norm(P, axis=1), 1.0, rtol=1e-6)
    f = synth.ndfd_features(3, 5000, P)
    np.testing.assert_allclose(np.linalg.norm(f, axis=1), 1.0, rtol=1e-5)
    own = (f @ P.T).max(1)
    q01, q50, q99 = np.quantile(own, [0.01, 0.5, 0.99])   # cos = 1/sqrt(1 + l^2), l ~ U[0.2, 3]
    assert 0.2 < q01 < 0.4 and 0.4 < q50 < 0.65 and 0.95 < q99 < 0.995
    gt = synth.ndfd_ground_truth(3, 0, 48, 72, P, block=24)
    np.testing.assert_allclose(np.linalg.norm(gt, axis=-1), 1.0, rtol=1e-5)
    lab = (gt @ P.T).argmax(-1)
    for by in range(2):
        for bx in range(3):
            blk = lab[24 * by:24 * by + 24, 24 * bx:24 * bx + 24]
            assert (blk == blk[0, 0]).all()
    cams = [dict(width=72, height=48)]
    df, dg = synth.ndfd_inputs_device(3, 4000, cams, D, torch.device("cpu"))
    assert df.dtype == torch.bfloat16 and dg.shape == (72 * 48, D)
    dfn = df.float().norm(dim=1)
    assert (dfn - 1).abs().max() < 1e-2
    dgl = dg.float().reshape(48, 72, D)
    sim = torch.einsum("hwd,hvd->hwv", dgl[:24, :24], dgl[:24, :24])   # pixels of one block share a prototype
    assert sim.mean() > 0.7
