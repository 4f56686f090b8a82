"""Parity of the NDFD losses and their backward (the CUDA path through the C
ABI) against the FP64 oracle.

Bars, for FP32 arithmetic over BF16 or FP32 inputs that the oracle reads
exactly:
  * L_gt and L_cf within 5e-5 absolute on every pixel with no threshold
    decision within 1e-5 relative of its edge (those pixels stay under 1%).
    The dot products f_gt . f_i and F . f_i carry an FP32 summation error of
    about sqrt(D) 2^-24 |a||b| (~1.4e-6 at D = 512); the activation's slope
    is at most k/4 = 5, and the weights sum to at most 1, so L_gt moves by
    ~7e-6; 5e-5 leaves a factor of seven.
  * Gradients of means, scales, quaternions and opacities within 1e-3
    relative L2 (the render backward's bar); SH gradients exactly zero.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2505_19154_gb300 import api, synth
from tests.helpers import MARGIN_TOL, check_margin_count, small_random_scene
from tests.test_gpu_parity import _t, check_grads

pytestmark = pytest.mark.gpu

L_TOL = 5e-5


def ndfd_case(n, seed, D, cams, bf16=True, sh_degree=1, spread=0.5):
    sc = small_random_scene(n, seed=seed, sh_degree=sh_degree, D=0, spread=spread)
    sc = {k: (np.asarray(v, np.float32) if isinstance(v, np.ndarray) else v) for k, v in sc.items()}
    protos = synth.ndfd_prototypes(seed, D)
    f = synth.ndfd_features(seed, n, protos)
    fg = [synth.ndfd_ground_truth(seed, v, c["height"], c["width"], protos) for v, c in enumerate(cams)]
    if bf16:
        f = synth.to_bf16(f)
        fg = [synth.to_bf16(x) for x in fg]
    sc["features"] = f
    return sc, fg


def tc_expected(D, bf16, path):
    """The tensor-core NDFD kernels take BF16 features with D in {256, 512}
    unless the FP32 path is asked for."""
    return bf16 and D in (256, 512) and path != api.PATH_FP32


def run_ndfd(sc, cams, prm, fg, bf16=True, grads=None, path=api.PATH_AUTO, save_state=False):
    dt = torch.bfloat16 if bf16 else torch.float32
    rast = api.Rasterizer(0, sh_degree=prm.get("sh_degree", 0), path=path)
    t = {k: _t(sc[k]) for k in ("means", "scales", "quats", "opacities", "sh")}
    feats = _t(sc["features"], dt)
    gt = _t(np.concatenate([x.reshape(-1, x.shape[-1]) for x in fg]), dt)
    rast.ctx.profile(True)
    st = rast.prepare(t["means"], t["scales"], t["quats"], t["opacities"], t["sh"], cams)
    nc = torch.empty(gt.shape[0], dtype=torch.int32, device=gt.device)
    Lgt, Lcf = rast.ndfd_forward(st, feats, gt, ncontrib=nc, save_state=save_state)
    out = dict(Lgt=Lgt.cpu().numpy(), Lcf=Lcf.cpu().numpy(), nc=nc.cpu().numpy())
    if save_state:
        out["state"] = {k: v.cpu().numpy() for k, v in st["ndfd_state"].items()}
    if grads is not None:
        g = rast.ndfd_backward(st, feats, gt, _t(grads[0]), _t(grads[1]))
        out["grads"] = {k: v.cpu().numpy() for k, v in g.items()}
    torch.cuda.synchronize()
    assert rast.ctx.sync_status() == api.OK
    prof = rast.ctx.profile_read()
    tc = tc_expected(int(sc["features"].shape[1]), bf16, path)
    assert ("ndfd_fwd_tc" if tc else "ndfd_fwd") in prof, prof
    if grads is not None:
        assert ("ndfd_bwd_tc" if tc else "ndfd_bwd") in prof, prof
    return out


def check_losses(out, sc, cams, prm, fg, prep):
    refs = oracle.ndfd_forward(sc, cams, prm, sc["features"], fg, prep=prep)
    rend = oracle.forward(sc, cams, prm, None, prep=prep)
    off = n_margin = n_pix = 0
    worst = 0.0
    for cam, ref, rr in zip(cams, refs, rend):
        P = cam["width"] * cam["height"]
        ok = rr["margin"].reshape(-1) > MARGIN_TOL
        n_margin += int((~ok).sum())
        n_pix += P
        for key in ("Lgt", "Lcf"):
            err = np.abs(out[key][off:off + P] - ref[key].reshape(-1))[ok].max(initial=0)
            worst = max(worst, err)
            assert err <= L_TOL, (key, err)
        np.testing.assert_array_equal(out["nc"][off:off + P][ok], ref["ncontrib"].reshape(-1)[ok])
        off += P
    check_margin_count(n_margin, n_pix, "NDFD")
    assert max(np.abs(r["Lcf"]).max() for r in refs) > 1e-2   # the case exercises L_cf
    return worst


@pytest.mark.parametrize("D,bf16,path", [(64, True, api.PATH_AUTO), (256, True, api.PATH_AUTO),
                                         (512, True, api.PATH_AUTO), (256, True, api.PATH_FP32),
                                         (512, True, api.PATH_FP32), (128, False, api.PATH_AUTO),
                                         (32, False, api.PATH_AUTO)])
def test_ndfd_forward_small(D, bf16, path):
    cams = [synth.look_at_camera(synth.ring_position(3.0, 20, 10), 64, 48)]
    sc, fg = ndfd_case(1500, 61 + D, D, cams, bf16=bf16)
    prm = dict(sh_degree=1)
    prep = oracle.prepare(sc, cams, prm)
    out = run_ndfd(sc, cams, prm, fg, bf16=bf16, path=path)
    worst = check_losses(out, sc, cams, prm, fg, prep)
    print(f"NDFD D={D} path={path}: worst loss error {worst:.3g}")


@pytest.mark.parametrize("D", [256, 512])
def test_ndfd_forward_tensor_core_ragged_multicamera_long_lists(D):
    """The tensor-core kernel over ragged cameras (partial tiles, both
    halves), lists of several 64-entry chunks, and a dense scene whose pixels
    stop early (the walk ends before the list does)."""
    cams = [synth.look_at_camera(synth.ring_position(2.4, a, e), w, h)
            for a, e, w, h in [(10, 5, 70, 50), (140, 25, 33, 47), (260, -20, 96, 64)]]
    sc, fg = ndfd_case(9000, 64 + D, D, cams, sh_degree=1, spread=0.45)
    prm = dict(sh_degree=1)
    prep = oracle.prepare(sc, cams, prm)
    out = run_ndfd(sc, cams, prm, fg, path=api.PATH_TC)
    worst = check_losses(out, sc, cams, prm, fg, prep)
    assert out["nc"].max() > 64   # some pixel's contributors span more than one chunk
    print(f"tensor-core NDFD D={D}: worst loss error {worst:.3g}, max contributors {out['nc'].max()}")


def test_ndfd_forward_multicamera_ragged():
    cams = [synth.look_at_camera(synth.ring_position(3.0, a, e), w, h)
            for a, e, w, h in [(0, 0, 70, 50), (130, 20, 33, 47), (250, -25, 96, 64)]]
    sc, fg = ndfd_case(4000, 62, 128, cams, sh_degree=2)
    prm = dict(sh_degree=2)
    prep = oracle.prepare(sc, cams, prm)
    out = run_ndfd(sc, cams, prm, fg)
    check_losses(out, sc, cams, prm, fg, prep)


@pytest.mark.parametrize("D,bf16,path", [(256, True, api.PATH_AUTO), (512, True, api.PATH_AUTO),
                                         (256, True, api.PATH_FP32), (512, True, api.PATH_FP32),
                                         (64, False, api.PATH_AUTO)])
def test_ndfd_backward_small(D, bf16, path):
    cams = [synth.look_at_camera(synth.ring_position(3.0, 40, -10), 64, 48)]
    sc, fg = ndfd_case(1500, 63 + D, D, cams, bf16=bf16, sh_degree=2)
    prm = dict(sh_degree=2)
    g = synth.rng(5, 4)
    a = g.standard_normal(64 * 48).astype(np.float32)
    b = g.standard_normal(64 * 48).astype(np.float32)
    prep = oracle.prepare(sc, cams, prm)
    out = run_ndfd(sc, cams, prm, fg, bf16=bf16, grads=(a, b), path=path)
    check_losses(out, sc, cams, prm, fg, prep)
    ref = oracle.ndfd_backward(sc, cams, prm, sc["features"], fg, [a], [b], prep=prep)
    check_grads(out["grads"], ref, keys=("means", "scales", "quats", "opacities"), tol=1e-3)
    assert not np.any(out["grads"]["sh"])
    # each loss alone (the two upstream gradients enter separately)
    z = np.zeros_like(a)
    for ga, gb in ((z, b), (a, z)):
        out2 = run_ndfd(sc, cams, prm, fg, bf16=bf16, grads=(ga, gb), path=path)
        ref2 = oracle.ndfd_backward(sc, cams, prm, sc["features"], fg, [ga], [gb], prep=prep)
        check_grads(out2["grads"], ref2, keys=("means", "scales", "quats", "opacities"), tol=1e-3)


@pytest.mark.parametrize("D", [256, 512])
def test_ndfd_backward_tensor_core_ragged_multicamera_long_lists(D):
    """The tensor-core backward over ragged cameras, walks of several
    64-entry chunks and pixels that stop early, against the oracle."""
    cams = [synth.look_at_camera(synth.ring_position(2.4, a, e), w, h)
            for a, e, w, h in [(10, 5, 70, 50), (140, 25, 33, 47), (260, -20, 96, 64)]]
    sc, fg = ndfd_case(9000, 65 + D, D, cams, sh_degree=1, spread=0.45)
    prm = dict(sh_degree=1)
    P = [c["width"] * c["height"] for c in cams]
    offs = np.cumsum([0] + P)
    g = synth.rng(7, 4)
    a = g.standard_normal(offs[-1]).astype(np.float32)
    b = g.standard_normal(offs[-1]).astype(np.float32)
    prep = oracle.prepare(sc, cams, prm)
    out = run_ndfd(sc, cams, prm, fg, grads=(a, b), path=api.PATH_TC)
    assert out["nc"].max() > 64
    ref = oracle.ndfd_backward(sc, cams, prm, sc["features"], fg, [a[offs[i]:offs[i + 1]] for i in range(3)],
                               [b[offs[i]:offs[i + 1]] for i in range(3)], prep=prep)
    check_grads(out["grads"], ref, keys=("means", "scales", "quats", "opacities"), tol=1e-3)


@pytest.mark.parametrize("D", [256, 512])
def test_ndfd_backward_from_saved_state(D):
    """The forward's saved end state (F_N, T after the walk, last
    contributor) in place of the backward's front-to-back rebuild: the state
    against the oracle's render of the same scene (F_N = sum w f, T_final,
    last) outside its margin pixels, and the gradients against the oracle
    and against the backward that rebuilds the state itself."""
    cams = [synth.look_at_camera(synth.ring_position(2.4, a, e), w, h)
            for a, e, w, h in [(10, 5, 70, 50), (140, 25, 33, 47), (260, -20, 96, 64)]]
    sc, fg = ndfd_case(9000, 65 + D, D, cams, sh_degree=1, spread=0.45)
    prm = dict(sh_degree=1)
    P = [c["width"] * c["height"] for c in cams]
    offs = np.cumsum([0] + P)
    g = synth.rng(8, 4)
    a = g.standard_normal(offs[-1]).astype(np.float32)
    b = g.standard_normal(offs[-1]).astype(np.float32)
    prep = oracle.prepare(sc, cams, prm)
    out = run_ndfd(sc, cams, prm, fg, grads=(a, b), path=api.PATH_TC, save_state=True)
    rebuilt = run_ndfd(sc, cams, prm, fg, grads=(a, b), path=api.PATH_TC)
    refs = oracle.forward(sc, cams, prm, sc["features"], prep=prep)
    state = out["state"]
    n_margin = 0
    for i, (cam, ref) in enumerate(zip(cams, refs)):
        sl = slice(offs[i], offs[i + 1])
        ok = ref["margin"].reshape(-1) > MARGIN_TOL
        n_margin += int((~ok).sum())
        np.testing.assert_array_equal(state["last"][sl][ok], ref["last"].reshape(-1)[ok])
        assert np.abs(state["T"][sl] - ref["T"].reshape(-1))[ok].max(initial=0) <= 1e-5
        F_ref = ref["feat"].reshape(-1, D)
        assert np.abs(state["F"][sl] - F_ref)[ok].max(initial=0) <= 1e-4 * max(1.0, np.abs(F_ref).max())
    check_margin_count(n_margin, int(offs[-1]), "NDFD state")
    ref = oracle.ndfd_backward(sc, cams, prm, sc["features"], fg, [a[offs[i]:offs[i + 1]] for i in range(3)],
                               [b[offs[i]:offs[i + 1]] for i in range(3)], prep=prep)
    check_grads(out["grads"], ref, keys=("means", "scales", "quats", "opacities"), tol=1e-3)
    for k in ("means", "scales", "quats", "opacities"):
        x, y = out["grads"][k].astype(np.float64), rebuilt["grads"][k].astype(np.float64)
        assert np.linalg.norm(x - y) <= 1e-5 * np.linalg.norm(y), k


def test_ndfd_backward_multicamera():
    cams = [synth.look_at_camera(synth.ring_position(3.0, a, e), w, h)
            for a, e, w, h in [(10, 5, 48, 40), (200, -15, 40, 56)]]
    sc, fg = ndfd_case(2500, 64, 128, cams, sh_degree=1)
    prm = dict(sh_degree=1)
    g = synth.rng(6, 4)
    P = sum(c["width"] * c["height"] for c in cams)
    a = g.standard_normal(P).astype(np.float32)
    b = g.standard_normal(P).astype(np.float32)
    prep = oracle.prepare(sc, cams, prm)
    out = run_ndfd(sc, cams, prm, fg, grads=(a, b))
    split = cams[0]["width"] * cams[0]["height"]
    ref = oracle.ndfd_backward(sc, cams, prm, sc["features"], fg, [a[:split], a[split:]], [b[:split], b[split:]],
                               prep=prep)
    check_grads(out["grads"], ref, keys=("means", "scales", "quats", "opacities"), tol=1e-3)


def test_ndfd_empty_scene_and_bad_arguments():
    cams = [synth.look_at_camera(synth.ring_position(3.0, 0, 0), 40, 24)]
    rast = api.Rasterizer(0, sh_degree=0)
    z = torch.zeros((0, 3), device="cuda")
    st = rast.prepare(z, z.clone() + 0.1, torch.zeros((0, 4), device="cuda"), torch.zeros(0, device="cuda"),
                      torch.zeros((0, 1, 3), device="cuda"), cams)
    feats = torch.zeros((0, 64), device="cuda", dtype=torch.bfloat16)
    gt = torch.ones((40 * 24, 64), device="cuda", dtype=torch.bfloat16)
    Lgt, Lcf = rast.ndfd_forward(st, feats, gt)
    assert not Lgt.any() and not Lcf.any()
    with pytest.raises(api.FhgsError) as e:
        rast.ndfd_forward(st, torch.zeros((0, 96), device="cuda", dtype=torch.bfloat16),
                          torch.ones((40 * 24, 96), device="cuda", dtype=torch.bfloat16))
    assert e.value.status == api.ERR_UNSUPPORTED
    big = torch.ones((40 * 24 * 64 + 8,), device="cuda", dtype=torch.bfloat16)
    with pytest.raises(api.FhgsError) as e:
        rast.ndfd_forward(st, feats, big[1:1 + 40 * 24 * 64].view(40 * 24, 64))
    assert e.value.status == api.ERR_ALIGNMENT
