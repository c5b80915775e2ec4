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
