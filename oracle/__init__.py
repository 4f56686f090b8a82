"""FP64 CPU oracle for the FHGS feature-splatting hot path (arXiv 2505.19154).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import or run this package.  It shares no
code with the CUDA library: the numeric work is in ``fhgs_oracle.c`` (plain C,
binary64, compiled here with gcc), and the per-tile lists are built with a
plain numpy sort.

Steps and the passages they follow:
  * ``bin_f32``      -- FP32 binning specification (pixel/tile rectangle,
                        depth key), App. A (CreateTiles, DuplicateWithKeys).
  * ``tile_lists``   -- 64-bit keys (tile id in the high word, depth bits in
                        the low word), one stable ascending sort, per-tile
                        [start, end) ranges, App. A (SortByKeys,
                        IdentifyTileRanges).
  * ``project``      -- EWA footprint + SH colour (Sec. 2.1 / App. A, the
                        3DGS rasterizer the paper builds on).
  * ``render``       -- Eq. 4 front to back, colour and feature (Sec. 3.1,
                        Sec. 3.2 DRF path).
  * ``render_bwd`` / ``project_bwd`` -- exact derivative of Eq. 4 with the
                        App. A.2 identity for dL/dalpha.
  * ``fuse``         -- compositing-weight-normalised fusion (Sec. 3.1).
  * ``splat_uv`` / ``render_2dgs_brute`` -- the surfel model of Sec. 3.1
                        (Eq. 1-3): ray-plane intersection u(x), G(u) and the
                        Eq. 4 compositing, per pixel over all surfels.
  * ``point_features`` -- the paper's point-to-feature assignment: a random
                        visible view, the nearest pixel, its feature (Sec. 3.1,
                        App. A "PointsFeatureFusion").
  * ``ndfd`` / ``ndfd_bwd`` -- the NDFD losses L_gt (Eq. 5) and L_cf (Eq. 6,
                        App. A.1) with the similarity activation of Sec. 3.3,
                        and their derivative through the weights w (Sec. 3.3,
                        App. A.2).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fhgs_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "libfhgs_oracle.so")

ORC_REC = 24
R_MX, R_MY, R_A, R_B, R_C, R_DEPTH, R_R, R_G, R_BL, R_RAW_R, R_RAW_G, R_RAW_B, R_VALID, R_OP = range(14)
R_SIG_A, R_SIG_B, R_SIG_C, R_EXT_X, R_EXT_Y = 14, 15, 16, 17, 18

DEFAULT_PARAMS = dict(znear=0.2, dilation=0.3, alpha_min=1.0 / 255.0, alpha_max=0.99,
                      t_eps=1e-4, cutoff_sq=9.0, fov_clamp=1.3, bg=(0.0, 0.0, 0.0),
                      tile=16, sh_degree=0)


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (OpenMP when available)."""
    if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= os.path.getmtime(_SRC):
        return _SO
    os.makedirs(_BUILD, exist_ok=True)
    base = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math"]
    tmp = _SO + f".tmp{os.getpid()}"
    try:
        subprocess.run(base + ["-fopenmp", _SRC, "-o", tmp, "-lm"], check=True,
                       capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base + [_SRC, "-o", tmp, "-lm"], check=True, capture_output=True)
    os.replace(tmp, _SO)
    return _SO


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        _lib.orc_num_threads.restype = ctypes.c_int
    return _lib


def num_threads() -> int:
    return int(lib().orc_num_threads())


def set_threads(n: int) -> None:
    lib().orc_set_threads(ctypes.c_int(int(n)))


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


def params_array(params: dict | None, dtype=np.float64) -> np.ndarray:
    p = dict(DEFAULT_PARAMS)
    if params:
        p.update(params)
    bg = tuple(p["bg"])
    return np.array([p["znear"], p["dilation"], p["alpha_min"], p["alpha_max"], p["t_eps"],
                     p["cutoff_sq"], p["fov_clamp"], bg[0], bg[1], bg[2], p["tile"],
                     p["sh_degree"]], dtype=dtype)


def camera_array(cam: dict, dtype=np.float64) -> np.ndarray:
    w2c = np.asarray(cam["w2c"], dtype=np.float64).reshape(3, 4)
    return np.concatenate([[cam["width"], cam["height"], cam["fx"], cam["fy"], cam["cx"],
                            cam["cy"]], w2c.reshape(-1)]).astype(dtype)


def sh_basis(dirs: np.ndarray):
    """Real SH basis Y (n, 16) and its gradient dY (n, 16, 3) at unit dirs."""
    d = _f64(dirs).reshape(-1, 3)
    Y = np.zeros((d.shape[0], 16))
    dY = np.zeros((d.shape[0], 16, 3))
    lib().orc_sh_basis(ctypes.c_int64(d.shape[0]), _p(d), _p(Y), _p(dY))
    return Y, dY


def quat_to_rot(q: np.ndarray) -> np.ndarray:
    q = _f64(q).reshape(-1, 4)
    R = np.zeros((q.shape[0], 3, 3))
    lib().orc_quat_to_rot(ctypes.c_int64(q.shape[0]), _p(q), _p(R))
    return R


def _k(scene) -> int:
    return int(np.asarray(scene["sh"]).reshape(len(scene["means"]), -1, 3).shape[1])


# --------------------------------------------------------------- projection
def project(scene: dict, cam: dict, params: dict | None = None) -> np.ndarray:
    """FP64 footprint + colour record per Gaussian, shape (n, ORC_REC)."""
    n = len(scene["means"])
    K = _k(scene)
    means, scales, quats = _f64(scene["means"]), _f64(scene["scales"]), _f64(scene["quats"])
    opac, sh = _f64(scene["opacities"]), _f64(scene["sh"])
    rec = np.zeros((n, ORC_REC))
    lib().orc_project(ctypes.c_int64(n), _p(means), _p(scales), _p(quats), _p(opac), _p(sh),
                      ctypes.c_int(K), _p(camera_array(cam)), _p(params_array(params)), _p(rec))
    return rec


def bin_f32(scene: dict, cam: dict, params: dict | None = None) -> dict:
    """FP32 binning specification for one camera."""
    n = len(scene["means"])
    means, scales, quats = _f32(scene["means"]), _f32(scene["scales"]), _f32(scene["quats"])
    pix = np.zeros((n, 4), np.int32)
    tile = np.zeros((n, 4), np.int32)
    ntiles = np.zeros(n, np.uint32)
    dbits = np.zeros(n, np.uint32)
    fp = np.zeros((n, 6), np.float32)
    lib().orc_bin_f32(ctypes.c_int64(n), _p(means), _p(scales), _p(quats),
                      _p(camera_array(cam, np.float32)), _p(params_array(params, np.float32)),
                      _p(pix), _p(tile), _p(ntiles), _p(dbits), _p(fp))
    return dict(pix=pix, tile=tile, ntiles=ntiles, dbits=dbits, fp=fp)


def tiles_xy(cam: dict, tile: int = 16):
    return (int(cam["width"]) + tile - 1) // tile, (int(cam["height"]) + tile - 1) // tile


def tile_lists(bins: list, cams: list, params: dict | None = None, tile_rect=None) -> dict:
    """Duplicate every Gaussian into the tiles of its rectangle, key it by
    (global tile id << 32 | depth bits), sort ascending with ties broken by
    Gaussian index, and find each tile's [start, end) range.

    The global tile id of camera c's tile (tx, ty) is
    cam_tile_offset[c] + ty * tiles_x(c) + tx.  ``tile_rect`` (tx0, ty0,
    tx1, ty1, inclusive; single camera only) restricts the lists to a
    window of tiles; other tiles get empty ranges."""
    tsz = int((params or {}).get("tile", 16))
    offs = [0]
    for c in cams:
        tx, ty = tiles_xy(c, tsz)
        offs.append(offs[-1] + tx * ty)
    keys_all, gids_all = [], []
    for ci, (b, cam) in enumerate(zip(bins, cams)):
        tx_n, _ = tiles_xy(cam, tsz)
        t = b["tile"].astype(np.int64)
        ok = b["ntiles"] > 0
        g = np.nonzero(ok)[0]
        t = t[ok]
        if tile_rect is not None:
            x0, y0, x1, y1 = tile_rect
            t = np.stack([np.maximum(t[:, 0], x0), np.maximum(t[:, 1], y0),
                          np.minimum(t[:, 2], x1), np.minimum(t[:, 3], y1)], 1)
            keep = (t[:, 0] <= t[:, 2]) & (t[:, 1] <= t[:, 3])
            g, t = g[keep], t[keep]
        w = t[:, 2] - t[:, 0] + 1
        h = t[:, 3] - t[:, 1] + 1
        cnt = w * h
        total = int(cnt.sum())
        rep = np.repeat(np.arange(len(g)), cnt)
        start = np.concatenate([[0], np.cumsum(cnt)[:-1]]).astype(np.int64)
        local = np.arange(total, dtype=np.int64) - start[rep]
        tx = t[rep, 0] + local % w[rep]
        ty = t[rep, 1] + local // w[rep]
        gt = offs[ci] + ty * tx_n + tx
        keys_all.append((gt.astype(np.uint64) << np.uint64(32)) | b["dbits"][g][rep].astype(np.uint64))
        gids_all.append(g[rep].astype(np.uint32))
    keys = np.concatenate(keys_all) if keys_all else np.zeros(0, np.uint64)
    gids = np.concatenate(gids_all) if gids_all else np.zeros(0, np.uint32)
    order = np.lexsort((gids, keys))
    keys, gids = keys[order], gids[order]
    ntot = offs[-1]
    tid = (keys >> np.uint64(32)).astype(np.int64)
    ranges = np.zeros((ntot, 2), np.uint32)
    if len(keys):
        bounds = np.nonzero(np.diff(tid))[0] + 1
        starts = np.concatenate([[0], bounds])
        ends = np.concatenate([bounds, [len(keys)]])
        ranges[tid[starts], 0] = starts
        ranges[tid[starts], 1] = ends
    return dict(keys=keys, gids=gids, ranges=ranges, cam_tile_offset=np.array(offs, np.int64))


# ------------------------------------------------------------------ render
def render(rec: np.ndarray, feats, gids, ranges_cam, cam: dict, params: dict | None = None,
           region=None) -> dict:
    """Tiled Eq. 4 render of `region` = (x0, y0, x1, y1) (default: image)."""
    W, H = int(cam["width"]), int(cam["height"])
    x0, y0, x1, y1 = region if region is not None else (0, 0, W, H)
    npx = (x1 - x0) * (y1 - y0)
    D = 0 if feats is None else int(np.asarray(feats).shape[1])
    f = _f64(feats) if D else None
    rgb = np.zeros((npx, 3))
    F = np.zeros((npx, D)) if D else None
    T = np.zeros(npx)
    last = np.zeros(npx, np.int32)
    margin = np.zeros(npx)
    nc = np.zeros(npx, np.int32)
    lib().orc_render(_p(rec), _p(f), ctypes.c_int(D), _p(np.ascontiguousarray(gids, np.uint32)),
                     _p(np.ascontiguousarray(ranges_cam, np.uint32)), _p(camera_array(cam)),
                     _p(params_array(params)), x0, y0, x1, y1, _p(rgb), _p(F), _p(T), _p(last),
                     _p(margin), _p(nc))
    hh, ww = y1 - y0, x1 - x0
    return dict(rgb=rgb.reshape(hh, ww, 3), feat=None if F is None else F.reshape(hh, ww, D),
                T=T.reshape(hh, ww), last=last.reshape(hh, ww), margin=margin.reshape(hh, ww),
                ncontrib=nc.reshape(hh, ww))


def render_brute(rec: np.ndarray, depth_key: np.ndarray, feats, cam: dict,
                 params: dict | None = None, region=None) -> dict:
    """Per-pixel brute force over all Gaussians sorted by (depth_key, index)."""
    W, H = int(cam["width"]), int(cam["height"])
    x0, y0, x1, y1 = region if region is not None else (0, 0, W, H)
    npx = (x1 - x0) * (y1 - y0)
    D = 0 if feats is None else int(np.asarray(feats).shape[1])
    f = _f64(feats) if D else None
    rgb = np.zeros((npx, 3))
    F = np.zeros((npx, D)) if D else None
    T = np.zeros(npx)
    margin = np.zeros(npx)
    sig = np.zeros(npx, np.uint64)
    lib().orc_render_brute(ctypes.c_int64(rec.shape[0]), _p(rec), _p(_f64(depth_key)), _p(f),
                           ctypes.c_int(D), _p(camera_array(cam)), _p(params_array(params)),
                           x0, y0, x1, y1, _p(rgb), _p(F), _p(T), _p(margin), _p(sig))
    hh, ww = y1 - y0, x1 - x0
    return dict(rgb=rgb.reshape(hh, ww, 3), feat=None if F is None else F.reshape(hh, ww, D),
                T=T.reshape(hh, ww), margin=margin.reshape(hh, ww), sig=sig.reshape(hh, ww))


def render_bwd(rec, feats, gids, ranges_cam, cam, params, region, dC, dF, want_feat=True) -> dict:
    """Per-Gaussian gradients of L = sum dC.rgb + dF.feat over `region`."""
    n = rec.shape[0]
    D = 0 if feats is None else int(np.asarray(feats).shape[1])
    f = _f64(feats) if D else None
    x0, y0, x1, y1 = region
    dC = _f64(dC).reshape(-1, 3)
    dFa = _f64(dF).reshape(-1, D) if (D and dF is not None) else None
    out = dict(mean2d=np.zeros((n, 2)), conic=np.zeros((n, 3)), op=np.zeros(n),
               rgb=np.zeros((n, 3)), feat=np.zeros((n, D)) if (D and want_feat) else None)
    lib().orc_render_bwd(_p(rec), _p(f), ctypes.c_int(D), _p(np.ascontiguousarray(gids, np.uint32)),
                         _p(np.ascontiguousarray(ranges_cam, np.uint32)), _p(camera_array(cam)),
                         _p(params_array(params)), x0, y0, x1, y1, _p(dC), _p(dFa),
                         _p(out["mean2d"]), _p(out["conic"]), _p(out["op"]), _p(out["rgb"]),
                         _p(out["feat"]))
    return out


def project_bwd(scene, cam, params, rec, g2d: dict) -> dict:
    n = len(scene["means"])
    K = _k(scene)
    out = dict(means=np.zeros((n, 3)), scales=np.zeros((n, 3)), quats=np.zeros((n, 4)),
               sh=np.zeros((n, K, 3)))
    lib().orc_project_bwd(ctypes.c_int64(n), _p(_f64(scene["means"])), _p(_f64(scene["scales"])),
                          _p(_f64(scene["quats"])), _p(_f64(scene["sh"])), ctypes.c_int(K),
                          _p(camera_array(cam)), _p(params_array(params)), _p(rec),
                          _p(_f64(g2d["mean2d"])), _p(_f64(g2d["conic"])), _p(_f64(g2d["rgb"])),
                          _p(out["means"]), _p(out["scales"]), _p(out["quats"]), _p(out["sh"]))
    return out


NDFD_K, NDFD_LAMBDA = 20.0, 0.5   # slope and threshold of the activation (Sec. 4)


def ndfd(rec, feats, gids, ranges_cam, cam, params, fgt, region=None, k=NDFD_K, lam=NDFD_LAMBDA) -> dict:
    """Per-pixel L_gt and L_cf of `region` (default: image); fgt is the
    region's ground-truth feature map, (h, w, D) or (h*w, D)."""
    W, H = int(cam["width"]), int(cam["height"])
    x0, y0, x1, y1 = region if region is not None else (0, 0, W, H)
    npx = (x1 - x0) * (y1 - y0)
    D = int(np.asarray(feats).shape[1])
    fg = _f64(fgt).reshape(npx, D)
    Lgt, Lcf, Wn = np.zeros(npx), np.zeros(npx), np.zeros(npx)
    nc = np.zeros(npx, np.int32)
    lib().orc_ndfd(_p(rec), _p(_f64(feats)), ctypes.c_int(D), _p(np.ascontiguousarray(gids, np.uint32)),
                   _p(np.ascontiguousarray(ranges_cam, np.uint32)), _p(camera_array(cam)),
                   _p(params_array(params)), x0, y0, x1, y1, _p(fg), ctypes.c_double(k),
                   ctypes.c_double(lam), _p(Lgt), _p(Lcf), _p(Wn), _p(nc))
    hh, ww = y1 - y0, x1 - x0
    return dict(Lgt=Lgt.reshape(hh, ww), Lcf=Lcf.reshape(hh, ww), W=Wn.reshape(hh, ww),
                ncontrib=nc.reshape(hh, ww))


def ndfd_bwd(rec, feats, gids, ranges_cam, cam, params, region, fgt, dLgt, dLcf, k=NDFD_K,
             lam=NDFD_LAMBDA) -> dict:
    """Footprint gradients of sum_p dLgt L_gt + dLcf L_cf over `region`
    (rgb is zero: colour does not enter the NDFD losses)."""
    n = rec.shape[0]
    D = int(np.asarray(feats).shape[1])
    x0, y0, x1, y1 = region
    npx = (x1 - x0) * (y1 - y0)
    out = dict(mean2d=np.zeros((n, 2)), conic=np.zeros((n, 3)), op=np.zeros(n), rgb=np.zeros((n, 3)))
    lib().orc_ndfd_bwd(_p(rec), _p(_f64(feats)), ctypes.c_int(D), _p(np.ascontiguousarray(gids, np.uint32)),
                       _p(np.ascontiguousarray(ranges_cam, np.uint32)), _p(camera_array(cam)),
                       _p(params_array(params)), x0, y0, x1, y1, _p(_f64(fgt).reshape(npx, D)),
                       ctypes.c_double(k), ctypes.c_double(lam), _p(_f64(dLgt).reshape(npx)),
                       _p(_f64(dLcf).reshape(npx)), _p(out["mean2d"]), _p(out["conic"]), _p(out["op"]))
    return out


def contributors(rec, gids, ranges_cam, cam, params, x: int, y: int, cap: int = 65536) -> dict:
    """The contributors of pixel (x, y) in compositing order: position in the
    tile's list, Gaussian id, alpha_i and T_i."""
    tsz = int((params or {}).get("tile", 16))
    tiles_x = (int(cam["width"]) + tsz - 1) // tsz
    t = (y // tsz) * tiles_x + x // tsz
    s, e = int(ranges_cam[t][0]), int(ranges_cam[t][1])
    lst = np.ascontiguousarray(np.asarray(gids, np.uint32)[s:e])
    pos = np.zeros(cap, np.int64)
    al, T = np.zeros(cap), np.zeros(cap)
    nc = lib().orc_contributors(_p(rec), _p(lst), ctypes.c_int64(e - s), _p(params_array(params)),
                                ctypes.c_double(x + 0.5), ctypes.c_double(y + 0.5), ctypes.c_int(cap),
                                _p(pos), _p(al), _p(T))
    nc = min(int(nc), cap)
    return dict(pos=pos[:nc], gid=lst[pos[:nc]].astype(np.int64), alpha=al[:nc], T=T[:nc])


# ------------------------------------------------------------- pipelines
def prepare(scene: dict, cams: list, params: dict | None = None, tile_rect=None, geometry: str = "fp64") -> dict:
    """Binning (FP32 spec), tile lists and FP64 records for every camera.

    geometry="fp32" composites over the FP32 binning specification's
    footprints (mean and conic rounded as that specification computes them)
    instead of the FP64 projection: every contribute/skip decision then
    rests on the same footprint as in an FP32 renderer that follows the
    specification, and only the compositing arithmetic stays FP64."""
    bins = [bin_f32(scene, c, params) for c in cams]
    lists = tile_lists(bins, cams, params, tile_rect=tile_rect)
    recs = [project(scene, c, params) for c in cams]
    if geometry == "fp32":
        for b, r in zip(bins, recs):
            fp = b["fp"].astype(np.float64)
            ok = b["ntiles"] > 0
            r[:, [R_MX, R_MY, R_A, R_B, R_C]] = np.where(ok[:, None], fp[:, :5], r[:, [R_MX, R_MY, R_A, R_B, R_C]])
            r[~ok, R_VALID] = 0.0
    elif geometry != "fp64":
        raise ValueError(geometry)
    return dict(bins=bins, lists=lists, recs=recs)


def _cam_ranges(lists: dict, ci: int) -> np.ndarray:
    o = lists["cam_tile_offset"]
    return np.ascontiguousarray(lists["ranges"][o[ci]:o[ci + 1]])


def forward(scene: dict, cams: list, params: dict | None = None, feats=None, region=None,
            prep: dict | None = None) -> list:
    """Render every camera (full image, or `region` for a single camera)."""
    prep = prep or prepare(scene, cams, params)
    outs = []
    for ci, cam in enumerate(cams):
        outs.append(render(prep["recs"][ci], feats, prep["lists"]["gids"], _cam_ranges(prep["lists"], ci),
                           cam, params, region))
    return outs


def backward(scene: dict, cams: list, params: dict | None, feats, dC_list, dF_list, region=None,
             prep: dict | None = None, want_feat=True) -> dict:
    """Gradients of sum_c (dC_c . rgb_c + dF_c . feat_c) with respect to
    means, scales, quats, opacities, sh and (optionally) features."""
    prep = prep or prepare(scene, cams, params)
    n = len(scene["means"])
    K = _k(scene)
    D = 0 if feats is None else int(np.asarray(feats).shape[1])
    tot = dict(means=np.zeros((n, 3)), scales=np.zeros((n, 3)), quats=np.zeros((n, 4)),
               opacities=np.zeros(n), sh=np.zeros((n, K, 3)),
               features=np.zeros((n, D)) if (D and want_feat) else None)
    for ci, cam in enumerate(cams):
        W, H = int(cam["width"]), int(cam["height"])
        reg = region if region is not None else (0, 0, W, H)
        g2 = render_bwd(prep["recs"][ci], feats, prep["lists"]["gids"], _cam_ranges(prep["lists"], ci),
                        cam, params, reg, dC_list[ci], None if dF_list is None else dF_list[ci],
                        want_feat=want_feat)
        gp = project_bwd(scene, cam, params, prep["recs"][ci], g2)
        for k in ("means", "scales", "quats", "sh"):
            tot[k] += gp[k]
        tot["opacities"] += g2["op"]
        if tot["features"] is not None:
            tot["features"] += g2["feat"]
    return tot


def fuse(scene: dict, views: list, maps: list, params: dict | None = None, prep: dict | None = None,
         margin_tol: float = 1e-5):
    """Fused per-Gaussian feature over all views.  maps[v]: (H, W, D).
    Also returns wflip: per Gaussian, a bound on the total weight a flipped
    near-threshold decision (within margin_tol) could move (orc_fuse_view)."""
    prep = prep or prepare(scene, views, params)
    n = len(scene["means"])
    D = int(np.asarray(maps[0]).shape[-1])
    num = np.zeros((n, D))
    den = np.zeros(n)
    wflip = np.zeros(n)
    for vi, cam in enumerate(views):
        W, H = int(cam["width"]), int(cam["height"])
        fm = _f64(maps[vi]).reshape(-1, D)
        lib().orc_fuse_view(_p(prep["recs"][vi]), _p(np.ascontiguousarray(prep["lists"]["gids"], np.uint32)),
                            _p(_cam_ranges(prep["lists"], vi)), _p(camera_array(cam)),
                            _p(params_array(params)), 0, 0, W, H, _p(fm), ctypes.c_int(D), _p(num),
                            _p(den), _p(wflip), ctypes.c_double(margin_tol))
    out = np.zeros((n, D))
    flag = np.zeros(n, np.int32)
    lib().orc_fuse_finalize(ctypes.c_int64(n), ctypes.c_int(D), _p(num), _p(den), _p(out), _p(flag))
    return dict(num=num, den=den, out=out, flag=flag, wflip=wflip)


def ndfd_forward(scene: dict, cams: list, params: dict | None, feats, fgt_list, prep: dict | None = None,
                 k=NDFD_K, lam=NDFD_LAMBDA) -> list:
    """Per-camera L_gt / L_cf maps (full images)."""
    prep = prep or prepare(scene, cams, params)
    return [ndfd(prep["recs"][ci], feats, prep["lists"]["gids"], _cam_ranges(prep["lists"], ci), cam, params,
                 fgt_list[ci], k=k, lam=lam) for ci, cam in enumerate(cams)]


def ndfd_backward(scene: dict, cams: list, params: dict | None, feats, fgt_list, dLgt_list, dLcf_list,
                  prep: dict | None = None, k=NDFD_K, lam=NDFD_LAMBDA) -> dict:
    """Gradients of sum_c sum_p (dLgt_c L_gt + dLcf_c L_cf) with respect to
    means, scales, quats and opacities (sh gets zeros; features are
    non-differentiable)."""
    prep = prep or prepare(scene, cams, params)
    n = len(scene["means"])
    K = _k(scene)
    tot = dict(means=np.zeros((n, 3)), scales=np.zeros((n, 3)), quats=np.zeros((n, 4)),
               opacities=np.zeros(n), sh=np.zeros((n, K, 3)))
    for ci, cam in enumerate(cams):
        W, H = int(cam["width"]), int(cam["height"])
        g2 = ndfd_bwd(prep["recs"][ci], feats, prep["lists"]["gids"], _cam_ranges(prep["lists"], ci), cam,
                      params, (0, 0, W, H), fgt_list[ci], dLgt_list[ci], dLcf_list[ci], k=k, lam=lam)
        gp = project_bwd(scene, cam, params, prep["recs"][ci], g2)
        for key in ("means", "scales", "quats", "sh"):
            tot[key] += gp[key]
        tot["opacities"] += g2["op"]
    return tot


def camera_array_f32(cam: dict) -> np.ndarray:
    """The camera as 18 binary32 values: width, height, fx, fy, cx, cy, [R|t]."""
    return camera_array(cam, np.float32)


def point_views(means, views: list, u, params: dict | None = None) -> dict:
    """Per point: the view drawn among those that see it (by u in [0, 1),
    -1 if none), the pixel index it projects to there, and how many views
    see it (binary32 projection spec)."""
    prm = dict(DEFAULT_PARAMS)
    prm.update(params or {})
    m = np.ascontiguousarray(means, np.float32).reshape(-1, 3)
    n = m.shape[0]
    cams = np.ascontiguousarray(np.concatenate([camera_array_f32(c) for c in views]), np.float32)
    uu = np.ascontiguousarray(u, np.float32).reshape(n)
    view = np.zeros(n, np.int32)
    pix = np.zeros(n, np.int32)
    cnt = np.zeros(n, np.int32)
    lib().orc_point_views_f32(ctypes.c_int64(n), _p(m), ctypes.c_int(len(views)), _p(cams),
                              ctypes.c_float(prm["znear"]), _p(uu), _p(view), _p(pix), _p(cnt))
    return dict(view=view, pixel=pix, count=cnt)


def point_features(means, views: list, maps: list, u, params: dict | None = None) -> dict:
    """Per point: the view drawn among those that see it (by u in [0, 1)),
    the pixel it projects to there, and that pixel's feature (zeros when no
    view sees it).  maps[v]: (H_v, W_v, D) or (H_v W_v, D)."""
    r = point_views(means, views, u, params)
    view, pix, cnt = r["view"], r["pixel"], r["count"]
    n = len(view)
    D = int(np.asarray(maps[0]).shape[-1])
    flat = [np.asarray(mp).reshape(-1, D) for mp in maps]
    out = np.zeros((n, D), np.float64)
    for i in np.nonzero(view >= 0)[0]:
        out[i] = flat[view[i]][pix[i]]
    return dict(features=out, view=view, pixel=pix, count=cnt)


# ------------------------------------------------------------ 2DGS surfels
def splat_uv(means, quats, scales2, cam: dict, px, py) -> dict:
    """Per (pixel centre, surfel) pair: the plane coordinates (u, v) of the
    pixel ray's intersection, its camera depth lambda, and whether the ray
    meets the plane at all."""
    mu = _f64(means).reshape(-1, 3)
    m = mu.shape[0]
    q = _f64(quats).reshape(m, 4)
    s2 = _f64(scales2).reshape(m, 2)
    u, v, lam = np.zeros(m), np.zeros(m), np.zeros(m)
    hit = np.zeros(m, np.int32)
    lib().orc_splat_uv(ctypes.c_int64(m), _p(mu), _p(q), _p(s2), _p(camera_array(cam)),
                       _p(_f64(px).reshape(m)), _p(_f64(py).reshape(m)), _p(u), _p(v), _p(lam), _p(hit))
    return dict(u=u, v=v, lam=lam, hit=hit.astype(bool))


def render_2dgs_brute(surfels: dict, cam: dict, params: dict | None = None, region=None) -> dict:
    """Brute-force surfel render (every pixel over every surfel, ordered by
    the centre's camera depth).  surfels: means [n,3], quats [n,4],
    scales2 [n,2] (s_u, s_v), opacities [n], rgb [n,3]."""
    W, H = int(cam["width"]), int(cam["height"])
    x0, y0, x1, y1 = region if region is not None else (0, 0, W, H)
    npx = (x1 - x0) * (y1 - y0)
    mu = _f64(surfels["means"]).reshape(-1, 3)
    n = mu.shape[0]
    w2c = np.asarray(cam["w2c"], np.float64).reshape(3, 4)
    depth = mu @ w2c[2, :3] + w2c[2, 3]
    rgb = np.zeros((npx, 3))
    T = np.zeros(npx)
    nc = np.zeros(npx, np.int32)
    lib().orc_render_2dgs_brute(ctypes.c_int64(n), _p(mu), _p(_f64(surfels["quats"]).reshape(n, 4)),
                                _p(_f64(surfels["scales2"]).reshape(n, 2)), _p(_f64(surfels["opacities"]).reshape(n)),
                                _p(_f64(surfels["rgb"]).reshape(n, 3)), _p(np.ascontiguousarray(depth)),
                                _p(camera_array(cam)), _p(params_array(params)), x0, y0, x1, y1, _p(rgb), _p(T),
                                _p(nc))
    hh, ww = y1 - y0, x1 - x0
    return dict(rgb=rgb.reshape(hh, ww, 3), T=T.reshape(hh, ww), ncontrib=nc.reshape(hh, ww))


def surfel_rect(means, quats, scales2, cam: dict, cut: float = 9.0) -> dict:
    """Screen bounding box (xmin, xmax, ymin, ymax) of each surfel's
    u^2 + v^2 <= cut ellipse, and whether it is bounded (the ellipse wholly
    in front of the camera; otherwise the box is the whole image)."""
    mu = _f64(means).reshape(-1, 3)
    n = mu.shape[0]
    rect = np.zeros((n, 4))
    bounded = np.zeros(n, np.int32)
    lib().orc_surfel_rect(ctypes.c_int64(n), _p(mu), _p(_f64(quats).reshape(n, 4)), _p(_f64(scales2).reshape(n, 2)),
                          _p(camera_array(cam)), ctypes.c_double(cut), _p(rect), _p(bounded))
    return dict(rect=rect, bounded=bounded.astype(bool))


def render_2dgs_bwd_brute(surfels: dict, cam: dict, params: dict | None, dC, region=None) -> dict:
    """Gradients of sum_p dC[p] . rgb[p] of render_2dgs_brute with respect
    to means, quats, scales2, opacities and rgb."""
    W, H = int(cam["width"]), int(cam["height"])
    x0, y0, x1, y1 = region if region is not None else (0, 0, W, H)
    mu = _f64(surfels["means"]).reshape(-1, 3)
    n = mu.shape[0]
    w2c = np.asarray(cam["w2c"], np.float64).reshape(3, 4)
    depth = mu @ w2c[2, :3] + w2c[2, 3]
    out = dict(means=np.zeros((n, 3)), quats=np.zeros((n, 4)), scales2=np.zeros((n, 2)), opacities=np.zeros(n),
               rgb=np.zeros((n, 3)))
    lib().orc_render_2dgs_bwd_brute(ctypes.c_int64(n), _p(mu), _p(_f64(surfels["quats"]).reshape(n, 4)),
                                    _p(_f64(surfels["scales2"]).reshape(n, 2)),
                                    _p(_f64(surfels["opacities"]).reshape(n)), _p(_f64(surfels["rgb"]).reshape(n, 3)),
                                    _p(np.ascontiguousarray(depth)), _p(camera_array(cam)), _p(params_array(params)),
                                    x0, y0, x1, y1, _p(_f64(dC).reshape(-1, 3)), _p(out["means"]), _p(out["quats"]),
                                    _p(out["scales2"]), _p(out["opacities"]), _p(out["rgb"]))
    return out


def bin_surfel_f32(means, quats, scales2, cam: dict, params: dict | None = None) -> dict:
    """The binary32 surfel binning rule: pixel and tile rectangles (x0, y0,
    x1, y1; inclusive), tile counts (0 = culled or off the image) and the
    depth key bits."""
    m = np.ascontiguousarray(means, np.float32).reshape(-1, 3)
    n = m.shape[0]
    pix = np.zeros((n, 4), np.int32)
    tile = np.zeros((n, 4), np.int32)
    nt = np.zeros(n, np.uint32)
    db = np.zeros(n, np.uint32)
    lib().orc_bin_surfel_f32(ctypes.c_int64(n), _p(m), _p(np.ascontiguousarray(quats, np.float32).reshape(n, 4)),
                             _p(np.ascontiguousarray(scales2, np.float32).reshape(n, 2)), _p(camera_array_f32(cam)),
                             _p(params_array(params, np.float32)), _p(pix), _p(tile), _p(nt), _p(db))
    return dict(pix=pix, tile=tile, ntiles=nt, dbits=db)


def render_2dgs(surfels: dict, cam: dict, params: dict | None = None, region=None, feats=None,
                tile_rect=None) -> dict:
    """Tiled surfel render: the binary32 binning rule, per-tile lists sorted
    by (tile, depth bits, id), and each pixel's walk of its tile's list.
    feats [n, D] (optional) are blended with the same weights.  Also returns
    each pixel's margin (decisions settling its contributor set)."""
    W, H = int(cam["width"]), int(cam["height"])
    x0, y0, x1, y1 = region if region is not None else (0, 0, W, H)
    npx = (x1 - x0) * (y1 - y0)
    mu = _f64(surfels["means"]).reshape(-1, 3)
    n = mu.shape[0]
    b = bin_surfel_f32(np.asarray(surfels["means"], np.float32), np.asarray(surfels["quats"], np.float32),
                       np.asarray(surfels["scales2"], np.float32), cam, params)
    lists = tile_lists([b], [cam], params, tile_rect=tile_rect)
    rgb = np.zeros((npx, 3))
    T = np.zeros(npx)
    nc = np.zeros(npx, np.int32)
    margin = np.zeros(npx)
    D = 0 if feats is None else int(np.asarray(feats).shape[1])
    fa = None if feats is None else _f64(feats).reshape(n, D)
    F = np.zeros((npx, D)) if feats is not None else None
    lib().orc_render_2dgs(_p(mu), _p(_f64(surfels["quats"]).reshape(n, 4)), _p(_f64(surfels["scales2"]).reshape(n, 2)),
                          _p(_f64(surfels["opacities"]).reshape(n)), _p(_f64(surfels["rgb"]).reshape(n, 3)),
                          _p(fa), ctypes.c_int(D), _p(np.ascontiguousarray(lists["gids"], np.uint32)),
                          _p(np.ascontiguousarray(_cam_ranges(lists, 0), np.uint32)), _p(camera_array(cam)),
                          _p(params_array(params)), x0, y0, x1, y1, _p(rgb), _p(F), _p(T), _p(nc), _p(margin))
    hh, ww = y1 - y0, x1 - x0
    return dict(rgb=rgb.reshape(hh, ww, 3), T=T.reshape(hh, ww), ncontrib=nc.reshape(hh, ww), bins=b, lists=lists,
                margin=margin.reshape(hh, ww), feat=None if F is None else F.reshape(hh, ww, D))


def splat_uv_T(means, quats, scales2, cam: dict, px, py) -> dict:
    """u(x), v(x) and the camera depth through the surfel's projective map
    T = K [a b c] and the two planes T_0 - x T_2, T_1 - y T_2."""
    mu = _f64(means).reshape(-1, 3)
    m = mu.shape[0]
    u, v, dep = np.zeros(m), np.zeros(m), np.zeros(m)
    lib().orc_splat_uv_T(ctypes.c_int64(m), _p(mu), _p(_f64(quats).reshape(m, 4)), _p(_f64(scales2).reshape(m, 2)),
                         _p(camera_array(cam)), _p(_f64(px).reshape(m)), _p(_f64(py).reshape(m)), _p(u), _p(v),
                         _p(dep))
    return dict(u=u, v=v, depth=dep)


def render_2dgs_bwd(surfels: dict, cam: dict, params: dict | None, dC, region=None, feats=None, dF=None,
                    tile_rect=None) -> dict:
    """Gradients of sum_p dC[p] . rgb[p] (+ dF[p] . feat[p] with features)
    of the tiled surfel render (render_2dgs) with respect to means, quats,
    scales2, opacities, rgb (and features)."""
    W, H = int(cam["width"]), int(cam["height"])
    x0, y0, x1, y1 = region if region is not None else (0, 0, W, H)
    mu = _f64(surfels["means"]).reshape(-1, 3)
    n = mu.shape[0]
    b = bin_surfel_f32(np.asarray(surfels["means"], np.float32), np.asarray(surfels["quats"], np.float32),
                       np.asarray(surfels["scales2"], np.float32), cam, params)
    lists = tile_lists([b], [cam], params, tile_rect=tile_rect)
    out = dict(means=np.zeros((n, 3)), quats=np.zeros((n, 4)), scales2=np.zeros((n, 2)), opacities=np.zeros(n),
               rgb=np.zeros((n, 3)))
    D = 0 if feats is None else int(np.asarray(feats).shape[1])
    fa = None if feats is None else _f64(feats).reshape(n, D)
    dFa = None if (feats is None or dF is None) else _f64(dF).reshape(-1, D)
    out["features"] = np.zeros((n, D)) if dFa is not None else None
    lib().orc_render_2dgs_bwd(ctypes.c_int64(n), _p(mu), _p(_f64(surfels["quats"]).reshape(n, 4)),
                              _p(_f64(surfels["scales2"]).reshape(n, 2)), _p(_f64(surfels["opacities"]).reshape(n)),
                              _p(_f64(surfels["rgb"]).reshape(n, 3)), _p(fa), ctypes.c_int(D), _p(dFa),
                              _p(np.ascontiguousarray(lists["gids"], np.uint32)),
                              _p(np.ascontiguousarray(_cam_ranges(lists, 0), np.uint32)), _p(camera_array(cam)),
                              _p(params_array(params)), x0, y0, x1, y1, _p(_f64(dC).reshape(-1, 3)),
                              _p(out["means"]), _p(out["quats"]), _p(out["scales2"]), _p(out["opacities"]),
                              _p(out["rgb"]), _p(out["features"]))
    return out


def _surfel_colour_scene(scene: dict) -> dict:
    """The surfels as a Gaussian scene for the colour record (SH along the
    view direction, + 0.5, clamped at 0): projection's colour depends only on
    the mean and SH; the third scale is a stand-in that nothing reads back."""
    s2 = _f64(scene["scales2"]).reshape(-1, 2)
    return dict(means=scene["means"], scales=np.concatenate([s2, s2[:, 1:]], axis=1), quats=scene["quats"],
                opacities=scene["opacities"], sh=scene["sh"], sh_degree=scene.get("sh_degree", 0))


def surfel_forward(scene: dict, cam: dict, params: dict | None = None, feats=None, region=None) -> dict:
    """Tiled surfel render of a surfel scene (means, quats, scales2,
    opacities, sh) with SH colour (and features [n, D] when given)."""
    prm = dict(params or {})
    prm["sh_degree"] = scene.get("sh_degree", 0)
    rec = project(_surfel_colour_scene(scene), cam, prm)
    surf = dict(means=scene["means"], quats=scene["quats"], scales2=scene["scales2"], opacities=scene["opacities"],
                rgb=rec[:, R_R:R_BL + 1])
    tr = None if region is None else (region[0] // 16, region[1] // 16, (region[2] - 1) // 16, (region[3] - 1) // 16)
    out = render_2dgs(surf, cam, prm, feats=feats, region=region, tile_rect=tr)
    out["rec"] = rec
    return out


def surfel_backward(scene: dict, cam: dict, params: dict | None, dC, feats=None, dF=None, region=None) -> dict:
    """Gradients of sum_p dC[p] . rgb[p] (+ dF[p] . feat[p]) of
    surfel_forward with respect to means (footprint and view direction),
    quats, scales2, opacities, sh (and features)."""
    prm = dict(params or {})
    prm["sh_degree"] = scene.get("sh_degree", 0)
    cs = _surfel_colour_scene(scene)
    rec = project(cs, cam, prm)
    surf = dict(means=scene["means"], quats=scene["quats"], scales2=scene["scales2"], opacities=scene["opacities"],
                rgb=rec[:, R_R:R_BL + 1])
    tr = None if region is None else (region[0] // 16, region[1] // 16, (region[2] - 1) // 16, (region[3] - 1) // 16)
    g = render_2dgs_bwd(surf, cam, prm, dC, feats=feats, dF=dF, region=region, tile_rect=tr)
    n = len(g["opacities"])
    gp = project_bwd(cs, cam, prm, rec, dict(mean2d=np.zeros((n, 2)), conic=np.zeros((n, 3)), rgb=g["rgb"]))
    return dict(means=g["means"] + gp["means"], quats=g["quats"], scales2=g["scales2"], opacities=g["opacities"],
                sh=gp["sh"], features=g["features"])


def ndfd_2dgs(surfels: dict, cam: dict, params: dict | None, feats, fgt, region=None, k=NDFD_K,
              lam=NDFD_LAMBDA) -> dict:
    """Per-pixel L_gt and L_cf over the tiled surfel render's contributors
    (the paper's NDFD on 2DGS geometry)."""
    W, H = int(cam["width"]), int(cam["height"])
    x0, y0, x1, y1 = region if region is not None else (0, 0, W, H)
    npx = (x1 - x0) * (y1 - y0)
    mu = _f64(surfels["means"]).reshape(-1, 3)
    n = mu.shape[0]
    D = int(np.asarray(feats).shape[1])
    b = bin_surfel_f32(np.asarray(surfels["means"], np.float32), np.asarray(surfels["quats"], np.float32),
                       np.asarray(surfels["scales2"], np.float32), cam, params)
    lists = tile_lists([b], [cam], params)
    Lgt, Lcf = np.zeros(npx), np.zeros(npx)
    nc = np.zeros(npx, np.int32)
    lib().orc_ndfd_2dgs(_p(mu), _p(_f64(surfels["quats"]).reshape(n, 4)), _p(_f64(surfels["scales2"]).reshape(n, 2)),
                        _p(_f64(surfels["opacities"]).reshape(n)), _p(np.ascontiguousarray(lists["gids"], np.uint32)),
                        _p(np.ascontiguousarray(_cam_ranges(lists, 0), np.uint32)), _p(camera_array(cam)),
                        _p(params_array(params)), x0, y0, x1, y1, _p(_f64(feats)), ctypes.c_int(D),
                        _p(_f64(fgt).reshape(npx, D)), ctypes.c_double(k), ctypes.c_double(lam), _p(Lgt), _p(Lcf),
                        _p(nc))
    hh, ww = y1 - y0, x1 - x0
    return dict(Lgt=Lgt.reshape(hh, ww), Lcf=Lcf.reshape(hh, ww), ncontrib=nc.reshape(hh, ww))


def ndfd_2dgs_bwd(surfels: dict, cam: dict, params: dict | None, feats, fgt, dLgt, dLcf, k=NDFD_K,
                  lam=NDFD_LAMBDA) -> dict:
    """Gradients of sum_p dLgt L_gt + dLcf L_cf of ndfd_2dgs (full image)
    with respect to means, quats, scales2 and opacities."""
    W, H = int(cam["width"]), int(cam["height"])
    npx = W * H
    mu = _f64(surfels["means"]).reshape(-1, 3)
    n = mu.shape[0]
    D = int(np.asarray(feats).shape[1])
    b = bin_surfel_f32(np.asarray(surfels["means"], np.float32), np.asarray(surfels["quats"], np.float32),
                       np.asarray(surfels["scales2"], np.float32), cam, params)
    lists = tile_lists([b], [cam], params)
    out = dict(means=np.zeros((n, 3)), quats=np.zeros((n, 4)), scales2=np.zeros((n, 2)), opacities=np.zeros(n))
    lib().orc_ndfd_2dgs_bwd(_p(mu), _p(_f64(surfels["quats"]).reshape(n, 4)), _p(_f64(surfels["scales2"]).reshape(n, 2)),
                            _p(_f64(surfels["opacities"]).reshape(n)),
                            _p(np.ascontiguousarray(lists["gids"], np.uint32)),
                            _p(np.ascontiguousarray(_cam_ranges(lists, 0), np.uint32)), _p(camera_array(cam)),
                            _p(params_array(params)), 0, 0, W, H, _p(_f64(feats)), ctypes.c_int(D),
                            _p(_f64(fgt).reshape(npx, D)), ctypes.c_double(k), ctypes.c_double(lam),
                            _p(_f64(dLgt).reshape(npx)), _p(_f64(dLcf).reshape(npx)), _p(out["means"]),
                            _p(out["quats"]), _p(out["scales2"]), _p(out["opacities"]))
    return out
