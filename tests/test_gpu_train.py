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
