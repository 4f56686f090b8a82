"""api.HostPipeline: host-resident inputs, copies overlapped with compute
across steps.  Its outputs must equal the direct calls on the same inputs
(forward bit for bit, gradients up to the order of the atomics)."""
import numpy as np
import pytest
import torch

from paper_2505_19154_gb300 import api, synth
from tests.test_gpu_tc import bf16_scene

pytestmark = pytest.mark.gpu


def test_host_pipeline_matches_direct_calls():
    dev = torch.device("cuda", 0)
    sc = bf16_scene(3000, seed=45, D=128, sh_degree=3)
    cams = [synth.look_at_camera(synth.ring_position(3.0, a, e), w, h)
            for a, e, w, h in [(20, 5, 80, 56), (200, -15, 48, 64)]]
    P = sum(c["width"] * c["height"] for c in cams)
    dC, dF = synth.upstream(11, P, 128)
    h = {k: torch.from_numpy(np.ascontiguousarray(sc[k], np.float32)) for k in
         ("means", "scales", "quats", "opacities", "sh")}
    h["features"] = torch.from_numpy(np.ascontiguousarray(sc["features"], np.float32)).to(torch.bfloat16)
    h["grad_rgb"] = torch.from_numpy(dC)
    h["grad_feat"] = torch.from_numpy(dF)
    h = {k: v.pin_memory() for k, v in h.items()}

    ref_r = api.Rasterizer(0, sh_degree=3, path=api.PATH_TC)
    d = {k: v.to(dev) for k, v in h.items()}
    st = ref_r.prepare(d["means"], d["scales"], d["quats"], d["opacities"], d["sh"], cams)
    rgb, feat = ref_r.forward(st, d["features"])
    grads = ref_r.backward(st, d["grad_rgb"], d["grad_feat"])
    ref = [rgb, feat] + [v for v in grads.values() if v is not None]
    ref = [r.cpu() for r in ref]

    rast = api.Rasterizer(0, sh_degree=3, path=api.PATH_TC)
    rast.prepare(d["means"], d["scales"], d["quats"], d["opacities"], d["sh"], cams)  # sizes the capacity
    pipe = api.HostPipeline(rast, cams, h)
    pipe.start()
    outs = [pipe.step() for _ in range(3)]
    pipe.finish()
    torch.cuda.synchronize()
    assert rast.ctx.sync_status() == api.OK
    bi, bo = pipe.bytes_per_step()
    assert bi == sum(v.numel() * v.element_size() for v in h.values())
    assert bo == sum(r.numel() * r.element_size() for r in ref)
    # steps 1 and 2 wrote different host buffers; step 0's buffer was reused by step 2
    for o in (outs[1], outs[2]):
        assert torch.equal(o[0], ref[0]) and torch.equal(o[1], ref[1])
        for a, b in zip(o[2:], ref[2:]):
            assert torch.linalg.norm((a - b).double()) <= 1e-5 * torch.linalg.norm(b.double()) + 1e-12
