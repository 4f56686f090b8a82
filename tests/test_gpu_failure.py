"""Failure detection on the GPU without a fault: every mbarrier wait of the
tensor-core kernels is bounded, and a wait that runs out latches
FHGS_ERR_TIMEOUT into the call's status word and ends the CTA.

fhgs_debug_wait_probe makes such a wait run out on purpose: each CTA first
waits, with a 0.2 ms limit, on an mbarrier that nothing arrives at, before
it has issued a copy or an MMA or allocated tensor memory.  The checks:
fhgs_sync_status reports FHGS_ERR_TIMEOUT for the render forward, the render
backward and the fusion; the status word is cleared by that read; and with
the probe off the same context renders again, equal to a render made before
the timeout (forward bit for bit, gradients within the order of their float
atomics).
"""
import numpy as np
import pytest
import torch

from paper_2505_19154_gb300 import api, synth
from tests.helpers import small_random_scene
from tests.test_gpu_parity import _t

pytestmark = pytest.mark.gpu

PROBE_NS = 200_000


def _case():
    sc = small_random_scene(1200, seed=61, sh_degree=1, D=128, spread=0.5)
    sc = {k: (np.asarray(v, np.float32) if isinstance(v, np.ndarray) else v) for k, v in sc.items()}
    cams = [synth.look_at_camera(synth.ring_position(3.0, 40, 10), 64, 48)]
    t = {k: _t(sc[k]) for k in ("means", "scales", "quats", "opacities", "sh")}
    feats = _t(synth.to_bf16(sc["features"]), torch.bfloat16)
    dC, dF = synth.upstream(6, 64 * 48, 128)
    return t, feats, cams, _t(dC), _t(dF)


def _grads(rast, st, dC, dF):
    g = rast.backward(st, dC, dF)
    return {k: v.clone() for k, v in g.items() if v is not None}


def test_wait_that_runs_out_is_reported_and_the_context_recovers():
    t, feats, cams, dC, dF = _case()
    rast = api.Rasterizer(0, sh_degree=1, path=api.PATH_TC)
    st = rast.prepare(t["means"], t["scales"], t["quats"], t["opacities"], t["sh"], cams)
    rgb0, feat0 = (x.clone() for x in rast.forward(st, feats))
    g0 = _grads(rast, st, dC, dF)
    torch.cuda.synchronize()
    assert rast.ctx.sync_status() == api.OK
    api.debug_wait_probe(PROBE_NS)
    try:
        rast.forward(st, feats)
        assert rast.ctx.sync_status() == api.ERR_TIMEOUT
        assert rast.ctx.sync_status() == api.OK  # the read cleared the word
        rast.backward(st, dC, dF)
        assert rast.ctx.sync_status() == api.ERR_TIMEOUT
        o, n_, d_ = rast.fuse(t["means"], t["scales"], t["quats"], t["opacities"], t["sh"], cams,
                              [torch.ones((64 * 48, 128), device=dC.device)])
        assert rast.ctx.sync_status() == api.ERR_TIMEOUT
    finally:
        api.debug_wait_probe(0)
    st = rast.prepare(t["means"], t["scales"], t["quats"], t["opacities"], t["sh"], cams)
    rgb1, feat1 = rast.forward(st, feats)
    g1 = _grads(rast, st, dC, dF)
    torch.cuda.synchronize()
    assert rast.ctx.sync_status() == api.OK
    assert torch.equal(rgb0, rgb1) and torch.equal(feat0, feat1)
    for k, v in g0.items():
        rel = (torch.linalg.norm((g1[k] - v).double()) / torch.linalg.norm(v.double()).clamp_min(1e-30)).item()
        assert rel <= 1e-5, (k, rel)
