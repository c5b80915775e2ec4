"""Template-row sharding of one registration over several processes.

Each rank owns a contiguous block of template rows and computes the 13
float64 partial sums of its rows: the total force F (3), the total weight W
and the moment T = sum_i f_i (Y_i - ybar)^T (9) (Eq. 5, Eq. 5.5, Eq. 6).  The
ranks all-gather the 13-vectors and add them in rank order, so every rank
obtains bit-identical totals, and every rank then applies the same pose
update (Eq. 5.5 - Eq. 12).  This is the method's only exchange: 13 doubles
per iteration.  The per-rank compute is a backend object with
``step_partials() -> ndarray[13]`` and ``step_apply(totals)``; the CUDA
backend (``CudaRowShard``) runs both in the scgr library.

``StreamShardedRegistration`` keeps the whole iteration on the device: the
backend writes its partial sums into a 13-double tensor
(``partials_into``), the ranks all-gather those tensors into a [world, 13]
tensor in rank order (NCCL on the GPU: enqueued on the same stream, no host
round trip), and the backend adds the rows in rank order and updates the pose
from the totals (``apply_parts``; on the GPU both halves are single
stream-ordered library calls).
"""
from __future__ import annotations

import numpy as np


def row_partition(m: int, world: int, rank: int):
    """Contiguous, balanced split of m rows: (row0, rows) of `rank`."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("bad rank/world")
    base, extra = divmod(m, world)
    row0 = rank * base + min(rank, extra)
    return row0, base + (1 if rank < extra else 0)


def reduce_partials(local13, group=None):
    """All-gather the ranks' 13-vectors and add them in rank order."""
    import torch
    import torch.distributed as dist
    v = np.asarray(local13, dtype=np.float64).reshape(13)
    if not (dist.is_available() and dist.is_initialized()):
        return v.copy()
    world = dist.get_world_size(group)
    dev = "cuda" if dist.get_backend(group) == "nccl" else "cpu"
    t = torch.from_numpy(v.copy()).to(dev)
    parts = [torch.zeros_like(t) for _ in range(world)]
    dist.all_gather(parts, t, group=group)
    total = np.zeros(13)
    for part in parts:                       # fixed order: rank 0, 1, ...
        total = total + part.cpu().numpy()
    return total


def gather_parts(local13, group=None):
    """All-gather the ranks' 13-vectors (tensors on the backend's device) into
    a [world, 13] tensor whose row r is rank r's (one process: [1, 13])."""
    import torch
    import torch.distributed as dist
    v = local13.reshape(13)
    if not (dist.is_available() and dist.is_initialized()):
        return v.reshape(1, 13)
    world = dist.get_world_size(group)
    if dist.get_backend(group) == "nccl":
        out = torch.empty((world, 13), dtype=v.dtype, device=v.device)
        dist.all_gather_into_tensor(out, v, group=group)
        return out
    parts = [torch.empty_like(v) for _ in range(world)]
    dist.all_gather(parts, v, group=group)
    return torch.stack(parts)


class StreamShardedRegistration:
    """Iterations of one row-sharded registration with the exchange kept on
    the backend's device: partials into a 13-double tensor, all-gather in
    rank order, rank-ordered totals and pose update by the backend."""

    def __init__(self, backend, group=None):
        self.backend = backend
        self.group = group
        self.buf = backend.new_partials_buffer()

    def run(self, iterations: int):
        for _ in range(iterations):
            self.backend.partials_into(self.buf)
            self.backend.apply_parts(gather_parts(self.buf, self.group))


class ShardedRegistration:
    """Runs iterations of one registration whose template rows are split
    over the ranks of `group` (default: the default process group)."""

    def __init__(self, backend, group=None):
        self.backend = backend
        self.group = group

    def run(self, iterations: int):
        for _ in range(iterations):
            local = self.backend.step_partials()
            self.backend.step_apply(reduce_partials(local, self.group))


class CudaRowShard:
    """Backend over one scgr context restricted to template rows
    [row0, row0 + rows) of the full template."""

    def __init__(self, X, Y0, row0: int, rows: int, params=None, stream=None):
        from . import scgr
        self.scgr = scgr
        self.ctx = scgr.scgr_create(params, stream)     # None: torch's current stream
        scgr.scgr_set_reference(self.ctx, X)
        scgr.scgr_set_template(self.ctx, Y0)
        scgr.scgr_set_row_range(self.ctx, row0, rows)
        scgr.scgr_compute_descriptors(self.ctx)

    def step_partials(self):
        return self.scgr.scgr_step_partials(self.ctx)

    def step_apply(self, totals):
        self.scgr.scgr_step_apply(self.ctx, totals)

    def new_partials_buffer(self):
        import torch
        return torch.empty(13, dtype=torch.float64, device="cuda")

    def partials_into(self, buf):
        self.scgr.scgr_step_partials_dev(self.ctx, buf)

    def apply_parts(self, parts):
        self.scgr.scgr_step_apply_dev(self.ctx, parts)

    def result(self):
        return self.scgr.scgr_get_result(self.ctx)

    def close(self):
        if self.ctx is not None:
            self.scgr.scgr_destroy(self.ctx)
            self.ctx = None
