"""View sharding across ranks, on the CPU with two gloo ranks.

The per-rank work here is done by the FP64 oracle (no GPU in these tests):
each rank fuses, or differentiates, only the views paper_2505_19154_gb300.shard
gives it, the per-Gaussian sums are combined with shard.allreduce_sum, and the
result must equal the single-process oracle over all views.
"""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle
from paper_2505_19154_gb300 import shard, synth
from tests.helpers import small_random_scene


def test_view_shard_partitions_every_view_once():
    for n in range(0, 13):
        for world in range(1, 6):
            got = [v for r in range(world) for v in shard.view_shard(n, r, world)]
            assert got == list(range(n))
            sizes = [len(shard.view_shard(n, r, world)) for r in range(world)]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        shard.view_shard(4, 2, 2)


def _views():
    return [synth.look_at_camera(synth.ring_position(2.5, a, e), w, h)
            for a, e, w, h in [(0, 0, 24, 20), (70, 15, 20, 24), (140, -10, 28, 16), (230, 25, 16, 16),
                               (300, -20, 24, 24)]]


def _maps(views, D):
    g = np.random.default_rng(5)
    return [g.normal(size=(v["height"], v["width"], D)) for v in views]


class _OracleRank:
    """Stands in for api.Rasterizer's fusion calls on a CPU rank."""

    def __init__(self, scene):
        self.scene = scene

    def fuse_accumulate(self, gaussians, views, maps, num, den):
        r = oracle.fuse(self.scene, list(views), [np.asarray(m, np.float64) for m in maps], dict(sh_degree=1))
        num += torch.from_numpy(r["num"])
        den += torch.from_numpy(r["den"])

    def fuse_finalize(self, gaussians, num, den, normalize):
        d = den[:, None]
        return torch.where(d > 0, num / torch.where(d > 0, d, torch.ones_like(d)), torch.zeros_like(num))


def _ndfd_inputs(views, D=8):
    protos = synth.ndfd_prototypes(33, D)
    feats = synth.ndfd_features(33, 60, protos).astype(np.float64)
    fgts = [synth.ndfd_ground_truth(33, v, c["height"], c["width"], protos, block=8) for v, c in enumerate(views)]
    g = np.random.default_rng(7)
    a = [g.normal(size=c["height"] * c["width"]) for c in views]
    b = [g.normal(size=c["height"] * c["width"]) for c in views]
    return feats, fgts, a, b


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        sc = small_random_scene(60, seed=31, sh_degree=1, D=0, spread=0.5)
        views = _views()
        D = 6
        maps = _maps(views, D)
        gauss = tuple(torch.from_numpy(np.asarray(sc[k], np.float64)) for k in
                      ("means", "scales", "quats", "opacities", "sh"))
        # fusion: num/den summed over ranks before the division
        fused, num, den = shard.fuse_sharded(_OracleRank(sc), gauss, views, lambda v: maps[v], D,
                                             dtype=torch.float64)
        # gradients of a multi-view step: per-rank backward of its views, one sum
        sc_f = dict(sc, features=np.random.default_rng(2).normal(size=(60, D)))
        mine = list(shard.view_shard(len(views), rank, world))
        ups = [synth.upstream(40 + v, views[v]["width"] * views[v]["height"], D) for v in range(len(views))]
        if mine:
            g = oracle.backward(sc_f, [views[v] for v in mine], dict(sh_degree=1), sc_f["features"],
                                [ups[v][0] for v in mine], [ups[v][1] for v in mine])
        else:
            g = {k: np.zeros_like(np.asarray(sc_f[k] if k != "opacities" else sc_f["opacities"], np.float64))
                 for k in ("means", "scales", "quats", "opacities", "sh", "features")}
        grads = {k: torch.from_numpy(np.ascontiguousarray(g[k], np.float64)) for k in
                 ("means", "scales", "quats", "opacities", "sh", "features")}
        shard.allreduce_sum(list(grads.values()))
        # NDFD gradients (L_gt, L_cf): the same per-rank backward and one sum
        nf, nfg, na, nb = _ndfd_inputs(views)
        if mine:
            gn = oracle.ndfd_backward(sc, [views[v] for v in mine], dict(sh_degree=1), nf, [nfg[v] for v in mine],
                                      [na[v] for v in mine], [nb[v] for v in mine])
        else:
            gn = {k: np.zeros_like(np.asarray(sc[k], np.float64)) for k in ("means", "scales", "quats", "opacities")}
        ngrads = {k: torch.from_numpy(np.ascontiguousarray(gn[k], np.float64))
                  for k in ("means", "scales", "quats", "opacities")}
        shard.allreduce_sum(list(ngrads.values()))
        if rank == 0:
            q.put(dict(fused=fused.numpy(), num=num.numpy(), den=den.numpy(),
                       grads={k: v.numpy() for k, v in grads.items()},
                       ndfd={k: v.numpy() for k, v in ngrads.items()}))
    finally:
        dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_gloo_ranks_match_single_process():
    oracle.build()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    try:
        res = q.get(timeout=240)
    finally:
        for p in procs:
            p.join(timeout=60)
            if p.is_alive():
                p.kill()
    assert all(p.exitcode == 0 for p in procs), [p.exitcode for p in procs]

    sc = small_random_scene(60, seed=31, sh_degree=1, D=0, spread=0.5)
    views = _views()
    D = 6
    maps = _maps(views, D)
    ref = oracle.fuse(sc, views, maps, dict(sh_degree=1))
    assert (ref["den"] > 0).sum() > 10  # the views see a good part of the scene
    np.testing.assert_allclose(res["num"], ref["num"], rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(res["den"], ref["den"], rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(res["fused"], ref["out"], rtol=1e-10, atol=1e-12)

    sc_f = dict(sc, features=np.random.default_rng(2).normal(size=(60, D)))
    ups = [synth.upstream(40 + v, views[v]["width"] * views[v]["height"], D) for v in range(len(views))]
    gref = oracle.backward(sc_f, views, dict(sh_degree=1), sc_f["features"], [u[0] for u in ups],
                           [u[1] for u in ups])
    for k, v in res["grads"].items():
        np.testing.assert_allclose(v, gref[k], rtol=1e-10, atol=1e-12, err_msg=k)

    nf, nfg, na, nb = _ndfd_inputs(views)
    nref = oracle.ndfd_backward(sc, views, dict(sh_degree=1), nf, nfg, na, nb)
    assert np.abs(nref["means"]).max() > 0
    for k, v in res["ndfd"].items():
        np.testing.assert_allclose(v, nref[k], rtol=1e-10, atol=1e-12, err_msg="ndfd " + k)
