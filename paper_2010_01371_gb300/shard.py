"""View-sharded data term of one reconstruction over several GPUs.

The PWLS data term (Eq. 3), its gradient (Eq. 5 at the current iterate) and
the separable curvature numerators (Eqs. 6, 8-11) are sums over rays; the rays
of a scan partition by view.  Each rank holds the whole image, the counts of
a contiguous block of views and a projector plan over those views only; it
computes its share with the library's kernels (``mbmd_objective``,
``mbmd_gradient``, ``mbmd_curvature`` on its plan), and one all-reduce (sum)
of the image-sized numerators -- plus one of the scalar objective -- gives
every rank the full quantities, in its own GPU memory.  The collective is
torch.distributed's (NCCL between GPUs); nothing here touches another GPU's
memory directly.

The view blocks are consecutive views of the same orbit, so a block's plan is
the full scan's geometry with angle0 advanced by the block's first view and
the same angular step: its rays are the full scan's rays of those views.
"""
from __future__ import annotations

import dataclasses


def view_partition(n_views: int, rank: int, world: int) -> tuple[int, int]:
    """Contiguous block (first view, number of views) of `rank`: the blocks
    of the `world` ranks cover every view once and differ in size by at most
    one view."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("rank must be in [0, world)")
    base, extra = divmod(n_views, world)
    v0 = rank * base + min(rank, extra)
    return v0, base + (1 if rank < extra else 0)


def view_subset_geometry(geom, v0: int, n: int):
    """The geometry of views [v0, v0 + n) of `geom` (any object with the
    mbir_geometry fields; dataclasses are copied, others get a shallow
    copy)."""
    step = geom.angle_span / geom.n_views
    fields = {"angle0": geom.angle0 + v0 * step, "angle_span": n * step, "n_views": n}
    if dataclasses.is_dataclass(geom):
        return dataclasses.replace(geom, **fields)
    import copy
    g = copy.copy(geom)
    for k, v in fields.items():
        setattr(g, k, v)
    return g


def rays_per_view(geom) -> int:
    return int(geom.n_u) * int(getattr(geom, "n_v", 1) or 1)


def view_subset_counts(y, geom, v0: int, n: int):
    """Columns of y ([n_chan][n_rays], rays in view order) of views
    [v0, v0 + n)."""
    r = rays_per_view(geom)
    return y[:, v0 * r:(v0 + n) * r]


class ViewShard:
    """One rank's share of the data term: plan over its views, spectrum and
    counts (device tensors).  `group` is a torch.distributed process group
    (None: the default group; no collective when the job has one rank, or
    with collective=False, which returns the share itself)."""

    def __init__(self, geom, Q, S, y, rank: int, world: int, group=None, n_mat_max: int = 8,
                 collective: bool = True):
        import paper_2010_01371_gb300 as p
        self.v0, self.n = view_partition(geom.n_views, rank, world)
        self.geom = view_subset_geometry(geom, self.v0, self.n)
        self.plan = p.Plan(self.geom, n_mat_max)
        self.spec = p.Spectrum(Q, S)
        self.y = view_subset_counts(y, geom, self.v0, self.n).contiguous()
        self.world, self.group = (world if collective else 1), group

    def _sum(self, t):
        if self.world > 1:
            import torch.distributed as dist
            dist.all_reduce(t, op=dist.ReduceOp.SUM, group=self.group)
        return t

    def objective(self, x):
        """L(x) of Eq. 3 over every view (device FP64 scalar, all-reduced)."""
        import paper_2010_01371_gb300 as p
        return self._sum(p.mbmd_objective(self.plan, self.spec, x, self.y))

    def gradient(self, x):
        """(grad L(x), L(x)): the numerator images A^T g of every view
        (all-reduced) and the objective."""
        import paper_2010_01371_gb300 as p
        g, obj = p.mbmd_gradient(self.plan, self.spec, x, self.y)
        return self._sum(g), self._sum(obj)

    def curvature(self, x):
        """The plain-SPS curvature numerators A^T kappa of every view
        (all-reduced)."""
        import paper_2010_01371_gb300 as p
        return self._sum(p.mbmd_curvature(self.plan, self.spec, x, self.y))
