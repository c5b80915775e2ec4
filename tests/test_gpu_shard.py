"""Template-row sharding on one GPU: two contexts each own half of the
template rows (two ranks emulated in one process; the host adds their
partial sums in rank order), and the result equals the unsharded run within
the pose tolerance while both "ranks" hold identical poses."""
import pytest
import torch

from paper_1902_01061_gb300 import scgr, shard, synth
from tests.gpu_helpers import Gpu, check_pose

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib(scgr_lib):
    return scgr_lib


def test_two_row_shards_match_unsharded_run():
    case = synth.mild(n=1500)
    iters = 12
    X = torch.from_numpy(case.X).cuda()
    Y0 = torch.from_numpy(case.Y0).cuda()
    params = scgr.scgr_default_params(E=iters)
    shards = [shard.CudaRowShard(X, Y0, *shard.row_partition(len(case.Y0), 2, r), params=params) for r in range(2)]
    try:
        for _ in range(iters):
            parts = [s.step_partials() for s in shards]
            total = parts[0] + parts[1]                 # rank order
            for s in shards:
                s.step_apply(total)
        a, b = (s.result() for s in shards)
    finally:
        for s in shards:
            s.close()
    assert list(a.R) == list(b.R) and list(a.t) == list(b.t) and a.s == b.s
    with Gpu(case.X, case.Y0, E=iters) as g:
        ref = g.run(iters)
    Ra, ta, sa = a.as_numpy()
    Rr, tr, sr = ref.as_numpy()
    diag = synth.bbox_diag(case.X)
    check_pose("two row shards vs unsharded", Ra, ta, sa, Rr, tr, sr, diag)


def test_stream_ordered_row_shards_match_unsharded_run():
    """The stream-ordered form: each shard enqueues its 13 partial sums into a
    device tensor, the tensors are gathered in rank order on the device (the
    all-gather of a multi-GPU run), and each shard adds them and updates its
    pose on the device; no host round trip per iteration.  Both shards hold
    identical poses, equal to the unsharded run within the pose tolerance."""
    case = synth.mild(n=1500)
    iters = 12
    X = torch.from_numpy(case.X).cuda()
    Y0 = torch.from_numpy(case.Y0).cuda()
    params = scgr.scgr_default_params(E=iters)
    shards = [shard.CudaRowShard(X, Y0, *shard.row_partition(len(case.Y0), 2, r), params=params) for r in range(2)]
    try:
        bufs = [s.new_partials_buffer() for s in shards]
        for _ in range(iters):
            for s, b in zip(shards, bufs):
                s.partials_into(b)
            parts = torch.stack(bufs)                   # rank order
            for s in shards:
                s.apply_parts(parts)
        a, b = (s.result() for s in shards)
    finally:
        for s in shards:
            s.close()
    assert list(a.R) == list(b.R) and list(a.t) == list(b.t) and a.s == b.s and a.iterations == iters
    with Gpu(case.X, case.Y0, E=iters) as g:
        ref = g.run(iters)
    Ra, ta, sa = a.as_numpy()
    Rr, tr, sr = ref.as_numpy()
    check_pose("two stream-ordered row shards vs unsharded", Ra, ta, sa, Rr, tr, sr, synth.bbox_diag(case.X))


def test_stream_ordered_entry_points_reject_bad_arguments():
    case = synth.mild(n=300)
    ctx = scgr.scgr_create(scgr.scgr_default_params(E=4))
    try:
        scgr.scgr_set_reference(ctx, torch.from_numpy(case.X).cuda())
        scgr.scgr_set_template(ctx, torch.from_numpy(case.Y0).cuda())
        scgr.scgr_compute_descriptors(ctx)
        lib = scgr.load()
        assert lib.scgr_step_partials_dev(ctx, None) == 1                  # NULL output
        parts = torch.zeros((1, 13), dtype=torch.float64, device="cuda")
        assert lib.scgr_step_apply_dev(ctx, parts.data_ptr(), 0) == 1      # no parts
        assert lib.scgr_step_apply_dev(ctx, None, 1) == 1                  # NULL parts
        buf = torch.zeros(13, dtype=torch.float64, device="cuda")
        scgr.scgr_step_partials_dev(ctx, buf)                              # then a good step
        scgr.scgr_step_apply_dev(ctx, buf)
        assert scgr.scgr_get_result(ctx).iterations == 1
    finally:
        scgr.scgr_destroy(ctx)


def test_row_range_guards():
    case = synth.mild(n=300)
    ctx = scgr.scgr_create(scgr.scgr_default_params())
    try:
        scgr.scgr_set_reference(ctx, torch.from_numpy(case.X).cuda())
        scgr.scgr_set_template(ctx, torch.from_numpy(case.Y0).cuda())
        with pytest.raises(scgr.ScgrError):
            scgr.scgr_set_row_range(ctx, 250, 100)           # outside the template
        scgr.scgr_set_row_range(ctx, 0, 150)
        scgr.scgr_compute_descriptors(ctx)
        with pytest.raises(scgr.ScgrError) as e:
            scgr.scgr_run(ctx, 1)                              # must iterate stepwise
        assert e.value.status == 2
        with pytest.raises(scgr.ScgrError) as e:
            scgr.scgr_step_partials(ctx)                       # needs params.E > 0
        assert e.value.status == 2
        buf = torch.zeros(13, dtype=torch.float64, device="cuda")
        with pytest.raises(scgr.ScgrError) as e:
            scgr.scgr_step_partials_dev(ctx, buf)
        assert e.value.status == 2
        with pytest.raises(scgr.ScgrError) as e:
            scgr.scgr_step_apply_dev(ctx, buf)
        assert e.value.status == 2
    finally:
        scgr.scgr_destroy(ctx)


def _nccl_worker(port, iters, q):
    """One NCCL rank (world size 1) on the GPU: the row-split registration
    with the exchange through NCCL collectives - the stream-ordered form's
    all_gather_into_tensor and the host form's all_gather."""
    import os
    import numpy as np
    import torch
    import torch.distributed as dist
    from paper_1902_01061_gb300 import scgr, shard, synth
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    torch.cuda.set_device(0)
    dist.init_process_group("nccl", rank=0, world_size=1)
    try:
        case = synth.mild(n=1500)
        X = torch.from_numpy(case.X).cuda()
        Y0 = torch.from_numpy(case.Y0).cuda()
        params = scgr.scgr_default_params(E=iters)
        out = []
        for form in ("stream", "host"):
            be = shard.CudaRowShard(X, Y0, 0, len(case.Y0), params=params)
            try:
                if form == "stream":
                    shard.StreamShardedRegistration(be).run(iters)
                else:
                    shard.ShardedRegistration(be).run(iters)
                r = be.result()
                out.append((np.array(r.R[:]), np.array(r.t[:]), r.s, r.iterations))
            finally:
                be.close()
        q.put(("ok", out))
    except Exception as e:                      # reported to the parent test
        q.put(("error", repr(e)))
    finally:
        dist.destroy_process_group()


def test_nccl_exchange_single_rank():
    """The NCCL branches of the shard exchange (device all-gather into a
    [world, 13] tensor, and the host form's all-gather of 13-vectors) run
    on the GPU in a one-rank NCCL process group (a child process, so the
    group does not outlive the test); both give the unsharded pose."""
    import socket
    import torch.multiprocessing as mp
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    iters = 10
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    p = ctx.Process(target=_nccl_worker, args=(port, iters, q))
    p.start()
    status, out = q.get(timeout=600)
    p.join(timeout=120)
    assert status == "ok", out
    assert p.exitcode == 0
    case = synth.mild(n=1500)
    with Gpu(case.X, case.Y0, E=iters) as g:
        ref = g.run(iters)
    Rr, tr, sr = ref.as_numpy()
    for (R, t, s, it), form in zip(out, ("stream-ordered", "host")):
        assert it == iters
        check_pose(f"one NCCL rank, {form} exchange vs unsharded", R.reshape(3, 3), t, s, Rr, tr, sr,
                   synth.bbox_diag(case.X))
