"""Seeded synthetic inputs shaped like the FHGS workloads (arXiv 2505.19154).

This module only draws random numbers and builds camera poses; it holds none
of the splatting arithmetic, and both the CUDA path and the FP64 oracle take
its outputs as inputs.  The paper trains on DTU / Mip-NeRF 360 / Tanks and
Temples scenes with SAM image embeddings (Sec. 4); none of those are
available here, so these generators stand in for them with the distributions
below (all seeded with numpy's Philox generator).

Scenes (per Gaussian):
  * "uniform" -- means U[-1,1]^3, log-scales U[-4.5,-2.5].
  * "normal"  -- means N(0, 0.6^2) clipped to [-2,2]^3, log-scales U[-5,-2].
  quaternions: normalised N(0, I4) draws; opacity = sigmoid(N(0,1)).
  SH: degree 0 with DC coefficients U[-sqrt(pi), sqrt(pi)] (DC colours
  uniform in [0,1]), or degree >= 1 with every coefficient N(0, 0.2^2).
  Features: N(0,1) per channel.
Cameras: pinhole, OpenCV axes (x right, y down, z forward); world "down"
is +y.  A camera at distance r looks at the origin.
"""
from __future__ import annotations

import math
import numpy as np


def rng(seed: int, stream: int = 0) -> np.random.Generator:
    return np.random.Generator(np.random.Philox(key=int(seed) * 1000003 + int(stream)))


def look_at_camera(pos, width: int, height: int, hfov_deg: float = 60.0) -> dict:
    """Pinhole camera at `pos` looking at the origin, horizontal FoV."""
    pos = np.asarray(pos, np.float64)
    f = -pos / np.linalg.norm(pos)
    down = np.array([0.0, 1.0, 0.0])
    r = np.cross(down, f)
    if np.linalg.norm(r) < 1e-9:
        r = np.array([1.0, 0.0, 0.0])
    r /= np.linalg.norm(r)
    d = np.cross(f, r)
    R = np.stack([r, d, f])
    t = -R @ pos
    fx = (width / 2.0) / math.tan(math.radians(hfov_deg) / 2.0)
    return dict(width=int(width), height=int(height), fx=float(fx), fy=float(fx),
                cx=width / 2.0, cy=height / 2.0,
                w2c=np.concatenate([R, t[:, None]], 1).astype(np.float64))


def ring_position(radius: float, azimuth_deg: float, elevation_deg: float) -> np.ndarray:
    az, el = math.radians(azimuth_deg), math.radians(elevation_deg)
    return np.array([radius * math.cos(el) * math.sin(az), -radius * math.sin(el),
                     -radius * math.cos(el) * math.cos(az)])


def make_scene(n: int, seed: int, kind: str = "normal", sh_degree: int = 3, D: int = 0,
               feat_dtype=np.float32) -> dict:
    g = rng(seed, 1)
    if kind == "uniform":
        means = g.uniform(-1.0, 1.0, (n, 3))
        log_s = g.uniform(-4.5, -2.5, (n, 3))
    elif kind == "normal":
        means = np.clip(g.normal(0.0, 0.6, (n, 3)), -2.0, 2.0)
        log_s = g.uniform(-5.0, -2.0, (n, 3))
    else:
        raise ValueError(kind)
    q = g.normal(0.0, 1.0, (n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    opac = 1.0 / (1.0 + np.exp(-g.normal(0.0, 1.0, n)))
    K = (sh_degree + 1) ** 2
    if sh_degree == 0:
        sh = g.uniform(-math.sqrt(math.pi), math.sqrt(math.pi), (n, 1, 3))
    else:
        sh = g.normal(0.0, 0.2, (n, K, 3))
    scene = dict(means=means.astype(np.float32), scales=np.exp(log_s).astype(np.float32),
                 quats=q.astype(np.float32), opacities=opac.astype(np.float32),
                 sh=sh.astype(np.float32), sh_degree=sh_degree)
    if D:
        f = rng(seed, 2).standard_normal((n, D), dtype=np.float32)
        scene["features"] = to_bf16(f) if feat_dtype == "bf16" else f
    return scene


def to_bf16(x: np.ndarray) -> np.ndarray:
    """Round float32 to the nearest bfloat16 (ties to even); returned as the
    float32 values of those bfloat16 numbers."""
    u = np.ascontiguousarray(x, np.float32).view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000).astype(np.uint32)
    return r.view(np.float32)


def upstream(seed: int, npx: int, D: int):
    """Upstream gradients dL/drgb (npx, 3) and dL/dfeat (npx, D), N(0,1)."""
    g = rng(seed, 3)
    dC = g.standard_normal((npx, 3), dtype=np.float32)
    dF = g.standard_normal((npx, D), dtype=np.float32) if D else None
    return dC, dF


# ------------------------------------------------------------- workloads
def config1(seed: int = 0):
    """1,024 Gaussians, one 64x64 camera at distance 4, 60 deg FoV, D=16."""
    scene = make_scene(1024, seed, "uniform", sh_degree=0, D=16)
    cam = look_at_camera([0.0, 0.0, -4.0], 64, 64)
    return scene, [cam]


def config2(seed: int = 0):
    """100k Gaussians, one 512x512 view, SH degree 3, D=128."""
    scene = make_scene(100_000, seed, "normal", sh_degree=3, D=128)
    cam = look_at_camera([0.0, 0.0, -4.0], 512, 512)
    return scene, [cam]


def config3(seed: int = 0, n: int = 1_000_000, D: int = 512):
    """1M Gaussians, one 1920x1080 view, SH degree 3, D=512 bfloat16."""
    scene = make_scene(n, seed, "normal", sh_degree=3, D=D, feat_dtype="bf16")
    cam = look_at_camera([0.0, 0.0, -4.0], 1920, 1080)
    return scene, [cam]


CROP3 = (928, 508, 992, 572)   # the 64x64 crop of the 1080p view used for errors


def config4_cameras(seed: int = 0, n_cams: int = 16):
    g = rng(seed, 4)
    cams = []
    for i in range(n_cams):
        w = int(g.integers(640, 1601))
        h = int(g.integers(480, 901))
        el = float(g.uniform(-30.0, 30.0))
        cams.append(look_at_camera(ring_position(4.0, i * 360.0 / n_cams, el), w, h))
    return cams


def config4(seed: int = 0, n: int = 500_000, D: int = 256):
    scene = make_scene(n, seed, "normal", sh_degree=3, D=D, feat_dtype="bf16")
    return scene, config4_cameras(seed)


def config5(seed: int = 0, n: int = 3_000_000):
    """3M Gaussians (config-2 distributions, SH degree 3) and the 64 views of
    the fusion workload."""
    return make_scene(n, seed, "normal", sh_degree=3), config5_views(seed)


def config5_views(seed: int = 0, n_views: int = 64, width: int = 1280, height: int = 720):
    g = rng(seed, 5)
    return [look_at_camera(ring_position(4.0, i * 360.0 / n_views, float(g.uniform(-30.0, 30.0))),
                           width, height) for i in range(n_views)]


def smooth_feature_map(seed: int, view: int, height: int, width: int, D: int,
                       sigma: float = 8.0) -> np.ndarray:
    """N(0,1) noise, separable Gaussian blur (sigma px, radius 3 sigma,
    reflected border without repeating the edge sample), then L2-normalised
    per pixel.  (H, W, D) float32."""
    from scipy import ndimage
    g = rng(seed, 1000 + view)
    x = g.standard_normal((height, width, D), dtype=np.float32)
    r = int(math.ceil(3 * sigma))
    k = np.exp(-0.5 * (np.arange(-r, r + 1) / sigma) ** 2)
    k = (k / k.sum()).astype(np.float32)
    for axis in (0, 1):
        x = ndimage.correlate1d(x, k, axis=axis, mode="mirror")
    x /= np.maximum(np.linalg.norm(x, axis=-1, keepdims=True), 1e-12)
    return x.astype(np.float32)


# ------------------------------------------------------ NDFD inputs
def ndfd_prototypes(seed: int, D: int, n_proto: int = 8) -> np.ndarray:
    """n_proto random unit vectors (the 'objects' of a segmentation-like
    embedding), (n_proto, D) float32."""
    p = rng(seed, 2000).standard_normal((n_proto, D))
    return (p / np.linalg.norm(p, axis=1, keepdims=True)).astype(np.float32)


def ndfd_features(seed: int, n: int, protos: np.ndarray) -> np.ndarray:
    """Per-Gaussian unit features clustered around the prototypes: a random
    prototype plus isotropic noise of a random level (cosine to the prototype
    from about 0.98 down to about 0.3), L2-normalised.  (n, D) float32."""
    g = rng(seed, 2001)
    k, D = protos.shape
    lab = g.integers(0, k, n)
    lvl = g.uniform(0.2, 3.0, n) / math.sqrt(D)
    f = protos[lab] + lvl[:, None] * g.standard_normal((n, D))
    return (f / np.linalg.norm(f, axis=1, keepdims=True)).astype(np.float32)


def ndfd_ground_truth(seed: int, view: int, height: int, width: int, protos: np.ndarray,
                      block: int = 24, noise: float = 0.5) -> np.ndarray:
    """Ground-truth feature map: the image is cut into block x block regions,
    each labelled with a random prototype, plus per-pixel noise (relative
    level `noise`), L2-normalised.  (height, width, D) float32."""
    g = rng(seed, 3000 + view)
    k, D = protos.shape
    by, bx = (height + block - 1) // block, (width + block - 1) // block
    lab = g.integers(0, k, (by, bx))
    lab = np.repeat(np.repeat(lab, block, 0), block, 1)[:height, :width]
    f = protos[lab] + (noise / math.sqrt(D)) * g.standard_normal((height, width, D), dtype=np.float32)
    f /= np.linalg.norm(f, axis=-1, keepdims=True)
    return f.astype(np.float32)


def ndfd_inputs_device(seed: int, n: int, cams, D: int, dev, n_proto: int = 8, block: int = 24, noise: float = 0.5,
                       chunk: int = 1 << 17):
    """The NDFD input recipe (clustered unit features around n_proto random
    unit prototypes, cosine to the own prototype from ~0.98 to ~0.3; a
    ground-truth map of block x block regions each labelled with a prototype
    plus per-pixel noise, L2-normalised) generated on the device with torch,
    in row chunks, rounded to BF16: the full-size workload, too large to
    make on the host.  Returns (features [n, D], feat_gt [P, D])."""
    import torch
    gen = torch.Generator(device=dev)
    gen.manual_seed(7_000_003 * (seed + 1))
    protos = torch.randn((n_proto, D), generator=gen, device=dev)
    protos = protos / protos.norm(dim=1, keepdim=True)
    feats = torch.empty((n, D), dtype=torch.bfloat16, device=dev)
    for r0 in range(0, n, chunk):
        m = min(chunk, n - r0)
        lab = torch.randint(0, n_proto, (m,), generator=gen, device=dev)
        lvl = (torch.rand((m,), generator=gen, device=dev) * 2.8 + 0.2) / math.sqrt(D)
        f = protos[lab] + lvl[:, None] * torch.randn((m, D), generator=gen, device=dev)
        feats[r0:r0 + m] = (f / f.norm(dim=1, keepdim=True)).to(torch.bfloat16)
    maps = []
    for c in cams:
        h, w = c["height"], c["width"]
        by, bx = (h + block - 1) // block, (w + block - 1) // block
        lab = torch.randint(0, n_proto, (by, bx), generator=gen, device=dev)
        lab = lab.repeat_interleave(block, 0).repeat_interleave(block, 1)[:h, :w].reshape(-1)
        g = torch.empty((h * w, D), dtype=torch.bfloat16, device=dev)
        for r0 in range(0, h * w, chunk):
            m = min(chunk, h * w - r0)
            x = protos[lab[r0:r0 + m]] + (noise / math.sqrt(D)) * torch.randn((m, D), generator=gen, device=dev)
            g[r0:r0 + m] = (x / x.norm(dim=1, keepdim=True)).to(torch.bfloat16)
        maps.append(g)
    return feats, torch.cat(maps)
