"""fhgs_render_bwd_noalloc: the backward for callers that cannot allocate.

Some callers cannot call cudaMalloc (code inside a custom device allocator or
a memory pool's callback, plugin hosts that own every device allocation), so
the library offers this context-free variant whose scratch is a fixed device
array.  These checks run its tensor-core and FP32 paths through the C ABI and
compare each result with the regular fhgs_render_bwd on the same inputs,
within the gradient tolerance of the other parity tests (1e-3 relative L2),
on two calls in a row (the second call must not see the first one's
scratch, and must leave the device's free memory unchanged) and on a
smaller call after them.  A bounded wait that runs out inside the call is
reported by fhgs_noalloc_sync_status.  The file is named so that pytest
collects it last.
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


def _case(path, feat_dtype, n, cams, seed, dev):
    """A prepared view set and the regular entry point's gradients for it."""
    D = 128
    means, scales, q, opac, sh, feats = (torch.from_numpy(a).to(dev) for a in _scene(n, seed, D))
    feats = feats.to(feat_dtype)
    rast = api.Rasterizer(0, sh_degree=3, path=path)
    st = rast.prepare(means, scales, q, opac, sh, cams)
    rast.forward(st, feats)
    P = sum(c["width"] * c["height"] for c in cams)
    gen = torch.Generator(device=dev)
    gen.manual_seed(seed)
    dC = torch.randn((P, 3), generator=gen, device=dev)
    dF = torch.randn((P, D), generator=gen, device=dev)
    ref = rast.backward(st, dC, dF)
    torch.cuda.synchronize()
    assert rast.ctx.sync_status() == api.OK
    # the prepared state holds raw pointers only: keep the inputs alive with it
    return dict(rast=rast, st=st, feats=feats, D=D, n=n, dC=dC, dF=dF, ref=ref, keep=(means, scales, q, opac, sh))


def _noalloc(c, dev, check_free=False):
    out = _grads_like(c["n"], c["D"], dev)  # the caller's outputs, allocated before the call
    st = c["st"]
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info(dev)[0]
    status = api.render_bwd_noalloc(st["g"], st["proj"], st["bins"], c["feats"], c["D"], st["cams"], c["rast"].params,
                                    st["T"], st["last"], c["dC"], c["dF"], out)
    torch.cuda.synchronize()
    free1 = torch.cuda.mem_get_info(dev)[0]
    assert status == api.OK, status
    if check_free:  # the call itself took no device memory
        assert free1 == free0, (free0, free1)
    assert api.noalloc_sync_status() == api.OK
    return out


def _check(out, ref, what):
    for k in ("means", "scales", "quats", "opacities", "sh", "features"):
        assert torch.isfinite(out[k]).all(), (what, k)
        rel = _rel(out[k], ref[k])
        assert rel <= 1e-3, (what, k, rel)


@pytest.mark.parametrize("path,feat_dtype", [(api.PATH_TC, torch.bfloat16), (api.PATH_FP32, torch.float32)])
def test_noalloc_backward_matches_the_regular_entry_point(path, feat_dtype):
    _build.build()
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    cams = [synth.look_at_camera(synth.ring_position(3.0, a, e), w, h)
            for a, e, w, h in [(0, 5, 96, 64), (120, -10, 64, 80)]]
    big = _case(path, feat_dtype, 3000, cams, 5, dev)
    # two calls in a row on the same device array: the second must not see
    # the first one's scratch, and by then the module is loaded, so the call
    # must leave the device's free memory unchanged
    for call in range(2):
        _check(_noalloc(big, dev, check_free=call == 1), big["ref"], f"call {call}")
    # a smaller call after the larger one: fewer Gaussians, one camera
    small = _case(path, feat_dtype, 1000, [synth.look_at_camera(synth.ring_position(3.0, 200, 15), 48, 40)], 6, dev)
    _check(_noalloc(small, dev, check_free=True), small["ref"], "smaller call")


def test_noalloc_status_reports_a_wait_that_ran_out():
    """A tensor-core wait that runs out inside the allocation-free call (made
    to run out by fhgs_debug_wait_probe, before any copy or MMA is issued) is
    reported by fhgs_noalloc_sync_status, which clears it: the next call
    reports FHGS_OK and matches the regular entry point again."""
    _build.build()
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    cams = [synth.look_at_camera(synth.ring_position(3.0, 60, 0), 64, 48)]
    c = _case(api.PATH_TC, torch.bfloat16, 1500, cams, 8, dev)
    st = c["st"]
    out = _grads_like(c["n"], c["D"], dev)
    api.debug_wait_probe(200_000)
    try:
        status = api.render_bwd_noalloc(st["g"], st["proj"], st["bins"], c["feats"], c["D"], st["cams"],
                                        c["rast"].params, st["T"], st["last"], c["dC"], c["dF"], out)
        assert status == api.OK  # launched; the timeout is a device-side condition
        assert api.noalloc_sync_status() == api.ERR_TIMEOUT
    finally:
        api.debug_wait_probe(0)
    assert api.noalloc_sync_status() == api.OK
    _check(_noalloc(c, dev), c["ref"], "after the timeout")


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
