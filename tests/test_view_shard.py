"""View sharding of one reconstruction's data term (Eqs. 3, 5, 6: sums over
rays, partitioned by view): the partition, the view-subset geometries and the
all-reduce of the numerator images.

* CPU: the partition covers every view once; a subset's view angles are the
  full scan's; two gloo ranks each compute the FP64 oracle's gradient and
  curvature numerators and data term over their views and all-reduce them,
  which must give the full scan's (host logic of the sharded path).
* GPU: the library's numerator images and objective of every view subset
  (plans over the subsets) add up to those of the full scan (one device; the
  NCCL path between GPUs is the same torch.distributed call and is not
  measured on hardware here).
"""
import math
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

import synth
from paper_2010_01371_gb300 import shard


def test_view_partition_covers_every_view_once():
    for n_views in [1, 7, 90, 720]:
        for world in [1, 2, 3, 8]:
            blocks = [shard.view_partition(n_views, r, world) for r in range(world)]
            views = [v for v0, n in blocks for v in range(v0, v0 + n)]
            assert views == list(range(n_views))
            sizes = [n for _, n in blocks]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        shard.view_partition(10, 2, 2)


@pytest.mark.parametrize("geom", [synth.config1().geom, synth.config2(nx=64, n_views=90, n_u=111).geom,
                                  synth.config5(n=16, n_views=12, n_u=32, n_v=24, rays=False).geom])
def test_view_subset_geometry_keeps_the_rays(geom):
    full = geom.view_angles()
    for world in [2, 3]:
        for r in range(world):
            v0, n = shard.view_partition(geom.n_views, r, world)
            sub = shard.view_subset_geometry(geom, v0, n)
            assert sub.n_views == n
            assert np.allclose(sub.view_angles(), full[v0:v0 + n], rtol=0, atol=1e-13)
            assert sub.n_rays == n * shard.rays_per_view(geom)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch
    import torch.distributed as dist

    import oracle
    from oracle import model
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        oracle.build_c()
        prob = synth.config4_slice(nx=32, n_views=30, n_u=55)
        g = prob.geom
        v0, n = shard.view_partition(g.n_views, rank, world)
        A = oracle.Projector(shard.view_subset_geometry(g, v0, n))
        y = shard.view_subset_counts(prob.y, g, v0, n)
        x = 0.7 * prob.truth
        l = A.project(x)
        grad = torch.as_tensor(A.backproject(model.data_grad_l(prob.Q, prob.S, l, y)))
        gam = A.project(np.ones_like(x))
        curv = torch.as_tensor(A.backproject(model.curvature_numerator(prob.Q, prob.S, l, y, gam)))
        obj = torch.tensor([model.data_objective(prob.Q, prob.S, l, y)], dtype=torch.float64)
        for t in (grad, curv, obj):
            dist.all_reduce(t, op=dist.ReduceOp.SUM)
        out.put((rank, grad.numpy(), curv.numpy(), float(obj[0])))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2])
def test_two_rank_all_reduce_gives_the_full_scan(oracle_lib, world):
    from oracle import model
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted([q.get(timeout=300) for _ in procs], key=lambda t: t[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    prob = synth.config4_slice(nx=32, n_views=30, n_u=55)
    A = oracle_lib.Projector(prob.geom)
    x = 0.7 * prob.truth
    l = A.project(x)
    grad = A.backproject(model.data_grad_l(prob.Q, prob.S, l, prob.y))
    curv = A.backproject(model.curvature_numerator(prob.Q, prob.S, l, prob.y, A.project(np.ones_like(x))))
    obj = model.data_objective(prob.Q, prob.S, l, prob.y)
    for _, g, c, o in res:
        assert np.allclose(g, grad, rtol=1e-12, atol=1e-12 * np.abs(grad).max())
        assert np.allclose(c, curv, rtol=1e-12, atol=1e-12 * np.abs(curv).max())
        assert abs(o - obj) <= 1e-12 * abs(obj)


@pytest.mark.gpu
@pytest.mark.parametrize("case", ["c4_64_fan", "c5_16_cone"])
@pytest.mark.parametrize("world", [2, 3])
def test_gpu_view_shards_add_up(case, world):
    """The shards' numerator images (mbmd_gradient, mbmd_curvature) and data
    terms on view-subset plans sum to the full scan's on one plan."""
    import torch

    import paper_2010_01371_gb300 as p
    from _helpers import rel_l2, to_dev, to_host
    prob = (synth.config4_slice(nx=64, n_views=90, n_u=111) if case == "c4_64_fan"
            else synth.config5(n=16, n_views=12, n_u=32, n_v=24))
    x = to_dev(0.7 * prob.truth)
    y = to_dev(prob.y)
    plan, spec = p.Plan(prob.geom), p.Spectrum(prob.Q, prob.S)
    g_full, o_full = p.mbmd_gradient(plan, spec, x, y)
    c_full = p.mbmd_curvature(plan, spec, x, y)
    g_sum, c_sum, o_sum = torch.zeros_like(g_full), torch.zeros_like(c_full), 0.0
    for r in range(world):
        sh = shard.ViewShard(prob.geom, prob.Q, prob.S, y, r, world, collective=False)   # rank r's share
        g, o = sh.gradient(x)
        g_sum += g
        c_sum += sh.curvature(x)
        o_sum += float(o.item())
    assert rel_l2(to_host(g_sum), to_host(g_full)) < 1e-6
    assert rel_l2(to_host(c_sum), to_host(c_full)) < 1e-6
    assert abs(o_sum - float(o_full.item())) <= 1e-6 * abs(float(o_full.item()))
