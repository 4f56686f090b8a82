"""fhgs_render_bwd_noalloc: the backward for callers that cannot allocate.

Some callers cannot call cudaMalloc (code inside a custom device allocator or
a memory pool's callback, plugin hosts that own every device allocation), so
the library offers this context-free variant whose scratch is a fixed device
array.  These checks run its tensor-core and FP32 paths through the C ABI and
compare each result with the regular fhgs_render_bwd on the same inputs,
within the gradient tolerance of the other parity tests (1e-3 relative L2),
on two calls in a row (the second call must not see the first one's
scratch).  The file is named so that pytest collects it last.
"""
import numpy as np
import pytest
import torch

from paper_2505_19154_gb300 import _build, api, synth

pytestmark = pytest.mark.gpu


def _scene(n, seed, D):
    g = synth.rng(seed, 91)
    means = g.normal(0.0, 0.5, (n, 3)).astype(np.float32)
    scales = np.exp(g.uniform(-3.5, -2.0, (n, 3))).astype(np.float32)
    q = g.normal(0.0, 1.0, (n, 4)).astype(np.float32)
    opac = (1.0 / (1.0 + np.exp(-g.normal(0.0, 1.0, n)))).astype(np.float32)
    sh = g.normal(0.0, 0.3, (n, 16, 3)).astype(np.float32)
    feats = synth.to_bf16(g.normal(0.0, 1.0, (n, D)).astype(np.float32))
    return means, scales, q, opac, sh, feats


def _grads_like(n, D, dev):
    return dict(means=torch.empty((n, 3), device=dev), scales=torch.empty((n, 3), device=dev),
                quats=torch.empty((n, 4), device=dev), opacities=torch.empty(n, device=dev),
                sh=torch.empty((n, 16, 3), device=dev), features=torch.empty((n, D), device=dev))


def _rel(a, b):
    a, b = a.double().cpu().numpy().ravel(), b.double().cpu().numpy().ravel()
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30)


@pytest.mark.parametrize("path,feat_dtype", [(api.PATH_TC, torch.bfloat16), (api.PATH_FP32, torch.float32)])
def test_noalloc_backward_matches_the_regular_entry_point(path, feat_dtype):
    _build.build()
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    n, D = 3000, 128
    means, scales, q, opac, sh, feats = (torch.from_numpy(a).to(dev) for a in _scene(n, 5, D))
    feats = feats.to(feat_dtype)
    cams = [synth.look_at_camera(synth.ring_position(3.0, a, e), w, h)
            for a, e, w, h in [(0, 5, 96, 64), (120, -10, 64, 80)]]
    rast = api.Rasterizer(0, sh_degree=3, path=path)
    st = rast.prepare(means, scales, q, opac, sh, cams)
    rast.forward(st, feats)
    P = sum(c["width"] * c["height"] for c in cams)
    gen = torch.Generator(device=dev)
    gen.manual_seed(7)
    dC = torch.randn((P, 3), generator=gen, device=dev)
    dF = torch.randn((P, D), generator=gen, device=dev)

    ref = rast.backward(st, dC, dF)
    torch.cuda.synchronize()
    assert rast.ctx.sync_status() == api.OK
    for call in range(2):  # the second call reuses the same device array
        out = _grads_like(n, D, dev)
        status = api.render_bwd_noalloc(st["g"], st["proj"], st["bins"], feats, D, st["cams"], rast.params,
                                        st["T"], st["last"], dC, dF, out)
        torch.cuda.synchronize()
        assert status == api.OK, status
        for k in ("means", "scales", "quats", "opacities", "sh", "features"):
            assert torch.isfinite(out[k]).all(), (call, k)
            rel = _rel(out[k], ref[k])
            assert rel <= 1e-3, (call, k, rel)


def test_noalloc_rejects_sizes_beyond_its_array():
    _build.build()
    dev = torch.device("cuda", 0)
    api.lib()
    n = api.NOALLOC_MAX_ENTRIES + 1
    means = torch.zeros((n, 3), device=dev)
    quats = torch.zeros((n, 4), device=dev)
    g = api.gaussians_struct(means, means, quats, means[:, 0].contiguous(), means)
    cams = api.make_cameras([synth.look_at_camera([0.0, 0.0, -4.0], 32, 32)])
    params = api.make_params(sh_degree=0)
    ranges = torch.zeros((4, 2), dtype=torch.int32, device=dev)
    gids = torch.zeros(16, dtype=torch.int32, device=dev)
    cnt = torch.zeros(1, dtype=torch.int64, device=dev)
    bins = api.Bins(gids.data_ptr(), None, ranges.data_ptr(), cnt.data_ptr(), 16)
    proj = torch.zeros(256, dtype=torch.uint8, device=dev)
    T = torch.ones(32 * 32, device=dev)
    last = torch.zeros(32 * 32, dtype=torch.int32, device=dev)
    dC = torch.zeros((32 * 32, 3), device=dev)
    out = dict(means=means, scales=means, quats=quats, opacities=means[:, 0].contiguous(), sh=means, features=None)
    status = api.render_bwd_noalloc(g, proj, bins, None, 0, cams, params, T, last, dC, None, out)
    assert status == api.ERR_UNSUPPORTED
