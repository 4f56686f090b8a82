"""One training iteration of the paper's loop (App. A, Alg. 1 loop body): render
the sampled view, the L1 photometric loss, the NDFD losses L_gt and L_cf of
Sec. 3.3 (means over the pixels, weighted by lambda1 and lambda2), both
backward passes, and an Adam update of the raw Gaussian parameters (means,
log-scales, quaternions, opacity logits, SH; features frozen).  Densification
is not part of it.

The sequencing is host code over a backend with these calls, so that the
same step runs on the library (`LibraryBackend`, every step a kernel of
libfhgs.so) and on any other implementation of the interface:
  activate(raw) -> dict with the rasterizer's scales and opacities
  prepare(params, cam) -> state          (projection and binning)
  render(state) -> rgb [P, 3]
  l1(rgb, target) -> (loss, grad [P, 3])
  ndfd(state, features, feat_gt) -> (L_gt [P], L_cf [P])
  backward(state, grad_rgb) -> activated-parameter gradients
  ndfd_backward(state, features, feat_gt, a, b) -> activated-parameter gradients
  add(g1, g2) -> g1 + g2 (per key)
  adam(raw, grads, state, t, lr, beta1, beta2, eps) -> updates raw in place and
      returns the activated scales and opacities
"""
from __future__ import annotations

from typing import Sequence

GROUPS = ("means", "log_scales", "quats", "logit_opacities", "sh")
LR_DEFAULTS = (1.6e-4, 5e-3, 1e-3, 5e-2, 2.5e-3)


class TrainStep:
    """Holds the raw parameters, the frozen features and the Adam state; each
    call runs one iteration on one view and returns the loss terms of the
    parameters it started from."""

    def __init__(self, backend, raw: dict, sh_degree: int, features, lr: Sequence[float] = LR_DEFAULTS,
                 lam1: float = 1.0, lam2: float = 1.0, beta1: float = 0.9, beta2: float = 0.999, eps: float = 1e-15):
        self.be = backend
        self.raw = raw
        self.sh_degree = sh_degree
        self.features = features
        self.lr = tuple(float(x) for x in lr)
        self.lam1, self.lam2 = float(lam1), float(lam2)
        self.beta1, self.beta2, self.eps = beta1, beta2, eps
        self.t = 0
        self.adam_state = backend.adam_init(raw, sh_degree)
        self.act = backend.activate(raw)

    def params(self) -> dict:
        return dict(means=self.raw["means"], scales=self.act["scales"], quats=self.raw["quats"],
                    opacities=self.act["opacities"], sh=self.raw["sh"])

    def __call__(self, cam: dict, target_rgb, feat_gt) -> dict:
        be = self.be
        st = be.prepare(self.params(), cam)
        rgb = be.render(st)
        L_rgb, grad_rgb = be.l1(rgb, target_rgb)
        npx = int(cam["width"]) * int(cam["height"])
        L_gt_map, L_cf_map = be.ndfd(st, self.features, feat_gt)
        L_gt = be.total(L_gt_map) / npx
        L_cf = be.total(L_cf_map) / npx
        g = be.backward(st, grad_rgb)
        gn = be.ndfd_backward(st, self.features, feat_gt, self.lam1 / npx, self.lam2 / npx)
        grads = be.add(g, gn)
        self.t += 1
        self.act = be.adam(self.raw, grads, self.adam_state, self.t, self.lr, self.beta1, self.beta2, self.eps)
        return dict(total=L_rgb + self.lam1 * L_gt + self.lam2 * L_cf, rgb=L_rgb, gt=L_gt, cf=L_cf)


class LibraryBackend:
    """The backend on libfhgs.so: projection, binning, the render and NDFD
    kernels, the L1 loss and the fused Adam kernel on one device."""

    def __init__(self, device: int = 0, sh_degree: int = 0, **params):
        import torch
        from . import api
        self.api, self.torch = api, torch
        self.rast = api.Rasterizer(device, sh_degree=sh_degree, **params)
        self.dev = torch.device("cuda", device)
        self._up = {}

    def adam_init(self, raw, sh_degree):
        return self.api.adam_state(int(raw["means"].shape[0]), sh_degree, self.dev)

    def activate(self, raw):
        s, o = self.api.activate_gaussians(self.rast.ctx, raw["log_scales"], raw["logit_opacities"])
        return dict(scales=s, opacities=o)

    def prepare(self, params, cam):
        return self.rast.prepare(params["means"], params["scales"], params["quats"], params["opacities"],
                                 params["sh"], [cam])

    def render(self, st):
        rgb, _ = self.rast.forward(st, None)
        return rgb

    def l1(self, rgb, target):
        loss, grad = self.api.l1_loss(self.rast.ctx, rgb, target.reshape(rgb.shape))
        return loss, grad

    def ndfd(self, st, features, feat_gt):
        # keep the walk's end state for ndfd_backward of the same iteration
        return self.rast.ndfd_forward(st, features, feat_gt, save_state=True)

    def total(self, x):
        return self.api.sum_f32(self.rast.ctx, x)

    def backward(self, st, grad_rgb):
        return self.rast.backward(st, grad_rgb, None)

    def ndfd_backward(self, st, features, feat_gt, a, b):
        # the loss terms are pixel means, so the upstream gradients are the
        # constants lambda / P, filled once per (size, value) and reused
        P = feat_gt.shape[0]
        key = (P, a, b)
        if key not in self._up:
            self._up = {key: (self.torch.full((P,), a, device=self.dev), self.torch.full((P,), b, device=self.dev))}
        ua, ub = self._up[key]
        return self.rast.ndfd_backward(st, features, feat_gt, ua, ub)

    def add(self, g1, g2):
        # the Adam kernel adds the gradient sets itself
        return [g1, g2]

    def adam(self, raw, grads, state, t, lr, beta1, beta2, eps):
        n = int(raw["means"].shape[0])
        scales = self.torch.empty((n, 3), device=self.dev)
        opac = self.torch.empty(n, device=self.dev)
        self.api.adam_gaussians(self.rast.ctx, raw, grads, state, t, lr, self.rast.params.sh_degree, beta1, beta2,
                                eps, scales_out=scales, opac_out=opac)
        return dict(scales=scales, opacities=opac)
