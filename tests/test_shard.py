"""Template-row sharding (one registration over several ranks): the host
logic of paper_1902_01061_gb300.shard with world_size-2 gloo ranks on CPU.
Each rank's partial sums come from the FP64 oracle (test-side backend), the
shard module reduces them in rank order and both ranks apply the totals."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

import oracle as O
from paper_1902_01061_gb300 import shard, synth


class OracleRowShard:
    """Rank compute from the oracle: partial sums of rows [row0, row0+rows)."""

    def __init__(self, X, Y0, prm, row0, rows, E):
        self.X = np.asarray(X, np.float64)
        self.Y = np.asarray(Y0, np.float64).copy()
        self.prm, self.E, self.it = prm, E, 0
        self.rows = np.arange(row0, row0 + rows)
        self.desc = O.descriptors(X, Y0, prm)
        self.eX = O.cloud_stats(self.X)[2]

    def step_partials(self):
        return O.partial_sums(self.Y, self.X, self.desc, self.prm, self.rows)

    def step_apply(self, totals):
        self.Y, _ = O.update_from_totals(self.Y, totals, self.prm, self.it, self.E, self.eX)
        self.it += 1

    # the stream-ordered shape of the backend interface, on CPU tensors
    def new_partials_buffer(self):
        import torch
        return torch.zeros(13, dtype=torch.float64)

    def partials_into(self, buf):
        import torch
        buf.copy_(torch.from_numpy(self.step_partials()))

    def apply_parts(self, parts):
        total = np.zeros(13)
        for row in parts.numpy():                  # rank order
            total = total + row
        self.step_apply(total)


def test_update_from_totals_equals_step_once():
    case = synth.mild(n=250)
    prm = O.Params()
    desc = O.descriptors(case.X, case.Y0, prm)
    X = case.X.astype(np.float64)
    Y = case.Y0.astype(np.float64)
    eX = O.cloud_stats(X)[2]
    a, _ = O.step_once(Y, X, desc, prm, 3, 10, eX)
    halves = [np.arange(0, 100), np.arange(100, 250)]
    tot = sum(O.partial_sums(Y, X, desc, prm, r) for r in halves)
    b, _ = O.update_from_totals(Y, tot, prm, 3, 10, eX)
    np.testing.assert_allclose(b, a, atol=1e-12)


def test_row_partition_covers_rows_once():
    for m in (1, 7, 100, 1001):
        for world in (1, 2, 3, 8):
            if world > m:
                continue
            parts = [shard.row_partition(m, world, r) for r in range(world)]
            assert parts[0][0] == 0 and sum(r for _, r in parts) == m
            for (a0, ar), (b0, _) in zip(parts, parts[1:]):
                assert a0 + ar == b0


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, iters, q, stream_form=False):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        case = synth.mild(n=300)
        prm = O.Params(E=iters)
        row0, rows = shard.row_partition(len(case.Y0), world, rank)
        be = OracleRowShard(case.X, case.Y0, prm, row0, rows, iters)
        if stream_form:
            shard.StreamShardedRegistration(be).run(iters)
        else:
            shard.ShardedRegistration(be).run(iters)
        q.put((rank, be.Y))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("stream_form", [False, True])
def test_two_gloo_ranks_match_single_rank(stream_form):
    """Host-side exchange (totals added by the shard module) and the
    stream-ordered form (tensors all-gathered in rank order, totals added by
    the backend) give the same registration on both ranks."""
    iters = 5
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, iters, q, stream_form)) for r in range(2)]
    for p in procs:
        p.start()
    out = dict(q.get(timeout=300) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    np.testing.assert_array_equal(out[0], out[1])          # identical totals -> identical templates
    case = synth.mild(n=300)
    ref = O.register(case.X, case.Y0, O.Params(E=iters), iterations=iters)
    np.testing.assert_allclose(out[0], ref["Y"], atol=1e-10)


def test_register_from_partials_equals_register():
    """The row-block form of the iteration (used to spread the oracle's force
    pass over a process pool) gives the pose of the plain iteration."""
    case = synth.mild(n=400)
    prm = O.Params(p=2.0)
    desc = O.descriptors(case.X, case.Y0, prm)
    a = O.register(case.X, case.Y0, prm, iterations=15, desc=desc)
    blocks = np.array_split(np.arange(len(case.Y0)), 3)
    b = O.register_from_partials(case.X, case.Y0, prm, 15, desc, blocks)
    np.testing.assert_allclose(b["R"], a["R"], atol=1e-11)
    np.testing.assert_allclose(b["t"], a["t"], atol=1e-11)
    assert abs(b["s"] - a["s"]) <= 1e-12 * a["s"]
    np.testing.assert_allclose(b["Y"], a["Y"], atol=1e-10)
