"""Parity of the training-step kernels (the L1 photometric loss and the Adam
update of the raw Gaussian parameters) against the oracle of the training
iteration.  FP32 against FP64: the loss within 1e-5 relative (FP32 partial
sums), its gradient exactly (a sign over a count), the parameters after
three Adam steps within 1e-5 relative to their change."""
import numpy as np
import pytest
import torch

from oracle import train
from paper_2505_19154_gb300 import api

pytestmark = pytest.mark.gpu


def test_l1_loss_matches_oracle():
    dev = torch.device("cuda", 0)
    g = np.random.default_rng(1)
    a = g.normal(size=(1000003, 3)).astype(np.float32)
    b = g.normal(size=(1000003, 3)).astype(np.float32)
    b[:10] = a[:10]   # equal entries: zero gradient
    ctx = api.Context(0)
    loss, grad = api.l1_loss(ctx, torch.from_numpy(a).to(dev), torch.from_numpy(b).to(dev))
    torch.cuda.synchronize()
    L, d = train.rgb_l1(a.astype(np.float64), b.astype(np.float64), a.size)
    assert abs(loss.item() - L) <= 1e-5 * L
    np.testing.assert_array_equal(grad.cpu().numpy(), d.astype(np.float32))
    assert ctx.sync_status() == api.OK


def test_adam_gaussians_match_oracle():
    dev = torch.device("cuda", 0)
    g = np.random.default_rng(2)
    n, deg = 1001, 1
    K = (deg + 1) ** 2
    raw = dict(means=g.normal(size=(n, 3)), log_scales=g.uniform(-4, -1, (n, 3)), quats=g.normal(size=(n, 4)),
               logit_opacities=g.normal(size=n), sh=g.normal(size=(n, K, 3)))
    raw = {k: v.astype(np.float32).astype(np.float64) for k, v in raw.items()}
    lr = [1.6e-4, 5e-3, 1e-3, 5e-2, 2.5e-3]
    t_raw = {k: torch.from_numpy(v.astype(np.float32)).to(dev) for k, v in raw.items()}
    state = api.adam_state(n, deg, dev)
    scales = torch.empty((n, 3), device=dev)
    opac = torch.empty(n, device=dev)
    ctx = api.Context(0)
    ost = train.adam_init(raw)
    ref = raw
    for t in (1, 2, 3):
        ga = dict(means=g.normal(size=(n, 3)), scales=g.normal(size=(n, 3)) * 10, quats=g.normal(size=(n, 4)),
                  opacities=g.normal(size=n), sh=g.normal(size=(n, K, 3)))
        ga = {k: v.astype(np.float32).astype(np.float64) for k, v in ga.items()}
        tg = {k: torch.from_numpy(v.astype(np.float32)).to(dev) for k, v in ga.items()}
        api.adam_gaussians(ctx, t_raw, tg, state, t, lr, deg, eps=1e-15, scales_out=scales, opac_out=opac)
        ref = train.adam_step(ref, train.raw_grads(ref, ga), ost, t, dict(zip(train.GROUPS, lr)), eps=1e-15)
    torch.cuda.synchronize()
    assert ctx.sync_status() == api.OK
    for k in train.GROUPS:
        got = t_raw[k].cpu().numpy().astype(np.float64)
        moved = np.abs(ref[k] - raw[k]).max()
        assert np.abs(got - ref[k]).max() <= 1e-5 * max(moved, 1e-30) + 2e-7 * np.abs(ref[k]).max(), k
    np.testing.assert_allclose(scales.cpu().numpy(), np.exp(t_raw["log_scales"].cpu().numpy()), rtol=1e-6)
    np.testing.assert_allclose(opac.cpu().numpy(), 1 / (1 + np.exp(-t_raw["logit_opacities"].cpu().numpy())),
                               rtol=1e-6)


def test_train_step_on_the_library_matches_the_oracle_iteration():
    """Three iterations of the composed training step (App. A, Alg. 1 loop
    body; L = L_rgb + l1 L_gt + l2 L_cf, Sec. 3.3) with every arithmetic step
    in the library -- activation, render, L1, NDFD, both backward passes, the
    gradient sum and Adam inside the update kernel, the loss totals -- against
    the oracle's iteration.  Bars: each loss term within 1e-5 relative (FP32
    partial sums; 1e-7 absolute), and after every iteration each raw
    parameter group within 1e-3 relative L2 of the oracle's change of it
    (the gradient bar: FP32 against FP64 gradients enter Adam's m and v)."""
    from oracle import train as otrain
    from paper_2505_19154_gb300 import synth
    from paper_2505_19154_gb300.train import GROUPS, LibraryBackend, TrainStep
    from tests.helpers import small_random_scene
    import oracle

    dev = torch.device("cuda", 0)
    n, D, deg = 300, 32, 1
    sc = small_random_scene(n, seed=53, sh_degree=deg, D=0, spread=0.4)
    sc["opacities"] = np.clip(sc["opacities"], 0.1, 0.9)
    cam = synth.look_at_camera(synth.ring_position(2.5, 20, 10), 40, 32)
    protos = synth.ndfd_prototypes(53, D)
    feats = synth.ndfd_features(53, n, protos).astype(np.float32)
    fgt = synth.ndfd_ground_truth(53, 0, 32, 40, protos, block=8).astype(np.float32)
    target = (oracle.forward(sc, [cam], dict(sh_degree=deg))[0]["rgb"] + 0.05).astype(np.float32)
    raw0 = {k: v.astype(np.float32).astype(np.float64) for k, v in otrain.raw_from_scene(sc).items()}
    lr = (2e-3, 1e-2, 1e-2, 5e-2, 2e-2)
    lam1, lam2 = 0.7, 1.3

    be = LibraryBackend(0, sh_degree=deg)
    be.rast.ctx.profile(True)
    raw_d = {k: torch.from_numpy(v.astype(np.float32)).to(dev) for k, v in raw0.items()}
    step = TrainStep(be, raw_d, deg, torch.from_numpy(feats).to(dev), lr=lr, lam1=lam1, lam2=lam2)
    tgt_d = torch.from_numpy(target.reshape(-1, 3)).to(dev)
    fgt_d = torch.from_numpy(fgt.reshape(-1, D)).to(dev)

    ref_raw = {k: v.copy() for k, v in raw0.items()}
    ref_state = otrain.adam_init(ref_raw)
    for t in (1, 2, 3):
        got = step(cam, tgt_d, fgt_d)
        prev = ref_raw
        ref_raw, total, parts = otrain.train_step(ref_raw, ref_state, t, deg, [cam], [target.astype(np.float64)],
                                                  feats.astype(np.float64), [fgt.astype(np.float64)], lam1, lam2,
                                                  dict(zip(GROUPS, lr)))
        torch.cuda.synchronize()
        assert be.rast.ctx.sync_status() == api.OK
        for key, ref_v in (("rgb", parts["rgb"]), ("gt", parts["gt"]), ("cf", parts["cf"]), ("total", total)):
            v = float(got[key].item() if hasattr(got[key], "item") else got[key])
            assert abs(v - ref_v) <= 1e-5 * abs(ref_v) + 1e-7, (t, key, v, ref_v)
        for k in GROUPS:
            g = step.raw[k].double().cpu().numpy()
            change = np.linalg.norm(ref_raw[k] - prev[k])
            rel = np.linalg.norm(g - ref_raw[k]) / max(change, 1e-30)
            assert rel <= 1e-3, (t, k, rel)
    assert parts["gt"] > 0 and parts["cf"] > 0
    prof = be.rast.ctx.profile_read()
    for name in ("activate", "l1_loss", "sum", "adam", "ndfd_fwd", "ndfd_bwd"):
        assert name in prof, (name, prof)
