"""Batching form on the GPU: many registrations of uneven sizes in one call
(scgr_batch_run) give each pair the pose that a one-pair-per-call run gives,
within the pose tolerance (0.5 degrees, 1e-3 of the diagonal, 1e-5 relative
scale), and match the FP64 oracle on small pairs.  Graph replay of the batch
loop is bit-identical to eager launches."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_1902_01061_gb300 import scgr, synth
from tests.gpu_helpers import Gpu, check, pose_errors

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib(scgr_lib):
    return scgr_lib


def make_pairs(sizes, seed=5):
    rng = np.random.default_rng(seed)
    out = []
    for i, n in enumerate(sizes):
        surf = synth.EllipsoidUnion.random(rng, 3)
        X = surf.sample_surface(rng, n).astype(np.float32)
        R = synth.rotation_matrix(synth.random_unit(rng), float(rng.uniform(5, 40)))
        s = float(rng.uniform(0.8, 1.25))
        nout = int(0.1 * n) if i % 2 else 0
        Y = s * X.astype(np.float64) @ R + rng.uniform(-0.2, 0.2, 3)
        if nout:
            Y = np.concatenate([Y, rng.uniform(Y.min(0), Y.max(0), size=(nout, 3))])
        out.append((X, Y.astype(np.float32)))
    return out


def run_batch(pairs, iters, tuning=(), **prm):
    ctx = scgr.scgr_create(scgr.scgr_default_params(**prm))
    try:
        for key, value in tuning:
            scgr.scgr_set_tuning(ctx, key, value)
        ro = np.cumsum([0] + [len(x) for x, _ in pairs])
        to = np.cumsum([0] + [len(y) for _, y in pairs])
        Xc = torch.from_numpy(np.concatenate([x for x, _ in pairs])).cuda()
        Yc = torch.from_numpy(np.concatenate([y for _, y in pairs])).cuda()
        res = scgr.scgr_batch_run(ctx, ro, Xc, to, Yc, iters)
        launches = scgr.scgr_launch_count(ctx)
    finally:
        scgr.scgr_destroy(ctx)
    return res, launches


def close(a, b, diag, what, rot=0.5, t=1e-3, s=1e-5):
    """the pose tolerances, each error recorded by check()"""
    Ra, ta, sa = a.as_numpy()
    Rb, tb, sb = b.as_numpy() if hasattr(b, "as_numpy") else b
    er, et, es = pose_errors(Ra, ta, sa, Rb, tb, sb, diag)
    check(f"{what}: rotation (deg)", er, rot)
    check(f"{what}: translation / bbox diagonal", et, t)
    check(f"{what}: scale (relative)", es, s)
    return True


@pytest.mark.parametrize("p", [2.0, 1.0])
def test_batch_matches_single_pair_runs(p):
    pairs = make_pairs([600, 257, 1500, 16, 2100, 513, 90])
    iters = 25
    res, launches = run_batch(pairs, iters, p=p)
    assert len(res) == len(pairs)
    for (X, Y), r in zip(pairs, res):
        with Gpu(X, Y, p=p) as g:
            single = g.run(iters)
        assert r.iterations == iters
        assert close(r, single, synth.bbox_diag(X), f"batched vs one call per pair (p={p:g})")


def test_one_pair_batch_matches_single_run():
    pairs = make_pairs([1800], seed=21)
    res, _ = run_batch(pairs, 20, p=2.0)
    X, Y = pairs[0]
    with Gpu(X, Y, p=2.0) as g:
        single = g.run(20)
    assert len(res) == 1 and close(res[0], single, synth.bbox_diag(X), "one-pair batch vs single run")


def test_batch_matches_oracle_on_small_pairs():
    pairs = make_pairs([300, 140, 420], seed=9)
    iters = 20
    res, _ = run_batch(pairs, iters)
    for (X, Y), r in zip(pairs, res):
        o = O.register(X, Y, O.Params(), iterations=iters)
        assert close(r, (o["R"], o["t"], o["s"]), synth.bbox_diag(X), "batched pose vs oracle")


def test_batch_graph_replay_equals_eager():
    pairs = make_pairs([400, 1200, 33, 800], seed=13)
    a, la = run_batch(pairs, 15)
    b, lb = run_batch(pairs, 15, use_graph=1)
    assert la == lb
    for ra, rb in zip(a, b):
        assert list(ra.R) == list(rb.R) and list(ra.t) == list(rb.t) and ra.s == rb.s


@pytest.mark.parametrize("P,chunk,use_graph", [(1, 16, 0), (2, 3, 1), (2, 16, 1), (4, 3, 0), (4, 16, 1)])
def test_persistent_batch_kernel_is_bit_identical(P, chunk, use_graph):
    """The persistent batched force kernel (resident blocks taking work items
    from a queue) gives every pair the same bits as one block per item: an
    item's sums do not depend on which block takes it.  Uneven sizes, many
    more items than resident blocks in the chunk-3 case, and graph replay
    (the queue head is cleared before every launch)."""
    pairs = make_pairs([2600, 257, 16, 1900, 700, 3100, 90], seed=29)
    base = ((scgr.SCGR_TUNE_BATCH_P, P), (scgr.SCGR_TUNE_BATCH_CHUNK_TILES, chunk))
    a, la = run_batch(pairs, 12, tuning=base, p=2.0, use_graph=use_graph)
    b, lb = run_batch(pairs, 12, tuning=base + ((scgr.SCGR_TUNE_BATCH_PERSISTENT, 1),), p=2.0, use_graph=use_graph)
    assert la == lb
    for ra, rb in zip(a, b):
        assert list(ra.R) == list(rb.R) and list(ra.t) == list(rb.t) and ra.s == rb.s


@pytest.mark.parametrize("P", [0, 2, 4])
def test_batch_chunk_tuning_keeps_results_close(P):
    pairs = make_pairs([3000, 700], seed=17)
    a, _ = run_batch(pairs, 10, p=2.0)
    ctx = scgr.scgr_create(scgr.scgr_default_params(p=2.0))
    try:
        scgr.scgr_set_tuning(ctx, scgr.SCGR_TUNE_BATCH_CHUNK_TILES, 3)
        scgr.scgr_set_tuning(ctx, scgr.SCGR_TUNE_BATCH_P, P)
        scgr.scgr_set_tuning(ctx, scgr.SCGR_TUNE_FORCE_RSQRT, 1)       # p = 2 through rsqrt
        ro = np.cumsum([0] + [len(x) for x, _ in pairs])
        to = np.cumsum([0] + [len(y) for _, y in pairs])
        b = scgr.scgr_batch_run(ctx, ro, torch.from_numpy(np.concatenate([x for x, _ in pairs])).cuda(), to,
                                torch.from_numpy(np.concatenate([y for _, y in pairs])).cuda(), 10)
        with pytest.raises(scgr.ScgrError):
            scgr.scgr_set_tuning(ctx, scgr.SCGR_TUNE_BATCH_CHUNK_TILES, 0)
    finally:
        scgr.scgr_destroy(ctx)
    for (X, _), ra, rb in zip(pairs, a, b):
        assert close(ra, rb, synth.bbox_diag(X), f"batched, chunk 3 / P {P} / rsqrt vs defaults")


@pytest.mark.parametrize("use_graph", [0, 1])
def test_mixed_shape_batch_matches_single_pair_runs(use_graph):
    """The mixed batched pass (SCGR_TUNE_BATCH_P = 0): pairs whose templates
    fill 512-point blocks take 4 points x 128 threads with shared-memory sums,
    the others 2 points x 128 threads, in one launch.  Sizes on both sides of
    the choice (600 and 2,100 points take the 2-point shape, 2,000, 4,096 and
    5,200 the 4-point one), and a 16-point pair; every pair against a
    one-pair-per-call run of the same library, and replay against eager."""
    pairs = make_pairs([600, 2000, 5200, 4096, 2100, 16, 1300], seed=37)
    iters = 15
    res, la = run_batch(pairs, iters, tuning=((scgr.SCGR_TUNE_BATCH_P, 0),), p=2.0, use_graph=use_graph)
    for (X, Y), r in zip(pairs, res):
        with Gpu(X, Y, p=2.0) as g:
            single = g.run(iters)
        assert r.iterations == iters
        assert close(r, single, synth.bbox_diag(X), "mixed-shape batch vs one call per pair")
    if use_graph:
        eager, lb = run_batch(pairs, iters, tuning=((scgr.SCGR_TUNE_BATCH_P, 0),), p=2.0, use_graph=0)
        assert la == lb
        for ra, rb in zip(res, eager):
            assert list(ra.R) == list(rb.R) and list(ra.t) == list(rb.t) and ra.s == rb.s


def test_batch_rejects_bad_offsets():
    ctx = scgr.scgr_create(scgr.scgr_default_params())
    try:
        X = torch.zeros((40, 3), dtype=torch.float32, device="cuda")
        with pytest.raises(scgr.ScgrError) as e:
            scgr.scgr_batch_run(ctx, [0, 20, 40], X, [0, 30, 40], X, 3)    # second template has 10 < 16
        assert e.value.status == 1
        with pytest.raises(scgr.ScgrError):
            scgr.scgr_batch_run(ctx, [1, 40], X, [0, 40], X, 3)            # offsets must start at 0
    finally:
        scgr.scgr_destroy(ctx)


def test_full_size_batch_in_the_benchmark_configuration():
    """The benchmark's 512-pair batch (500-20,000 points per cloud, log-uniform;
    5.4 M points) at full size, in the launch configuration the benchmark's
    autotuner picks on GB300 (2 points per thread, 16-tile chunks, one CUDA
    graph), for 20 iterations: the three smallest pairs and the largest pair
    against the FP64 oracle, and three pairs (largest, median, one more)
    against one-pair-per-call runs of the same library."""
    pairs = synth.batch_case()
    iters = 20
    tuning = ((scgr.SCGR_TUNE_BATCH_P, 2), (scgr.SCGR_TUNE_BATCH_CHUNK_TILES, 16))
    res, launches = run_batch([(pp.X, pp.Y0) for pp in pairs], iters, tuning=tuning, p=2.0, use_graph=1)
    assert len(res) == len(pairs) and all(r.iterations == iters for r in res)
    sizes = np.array([len(pp.X) for pp in pairs])
    order = np.argsort(sizes, kind="stable")
    for i in order[:3]:
        pp = pairs[i]
        o = O.register(pp.X, pp.Y0, O.Params(p=2.0), iterations=iters)
        assert close(res[i], (o["R"], o["t"], o["s"]), synth.bbox_diag(pp.X), "full-size batch, smallest pairs vs oracle")
    for i in (order[-1], order[len(order) // 2], order[len(order) // 3]):
        pp = pairs[i]
        with Gpu(pp.X, pp.Y0, p=2.0) as g:
            single = g.run(iters)
        assert close(res[i], single, synth.bbox_diag(pp.X), "full-size batch vs one call per pair")
    # the largest pair against the FP64 oracle as well, its force rows spread
    # over a spawned process pool (row blocks added in block order)
    import multiprocessing as mp
    import os
    pp = pairs[order[-1]]
    prm = O.Params(p=2.0)
    d = O.descriptors(pp.X, pp.Y0, prm)
    slim = {"aX": d["aX"], "aY": d["aY"], "sigma": d["sigma"]}
    workers = max(1, min(16, os.cpu_count() or 1))
    blocks = np.array_split(np.arange(len(pp.Y0)), workers)
    with mp.get_context("spawn").Pool(workers) as pool:
        o = O.register_from_partials(pp.X, pp.Y0, prm, iters, slim, blocks, map_partials=pool.map)
    assert close(res[order[-1]], (o["R"], o["t"], o["s"]), synth.bbox_diag(pp.X),
                 f"full-size batch, largest pair ({len(pp.X):,} x {len(pp.Y0):,}) vs oracle")


def test_batch_with_g_equals_s_matches_single_pair_runs():
    """The batched form with the g = s weighting of Sec. IV (mixed shapes):
    every pair against a one-pair-per-call run of the same parameters."""
    pairs = make_pairs([900, 2100, 400, 3300], seed=43)
    iters = 15
    res, _ = run_batch(pairs, iters, tuning=((scgr.SCGR_TUNE_BATCH_P, 0),), p=2.0, g_mode=0)
    for (X, Y), r in zip(pairs, res):
        with Gpu(X, Y, p=2.0, g_mode=0) as g:
            single = g.run(iters)
        assert close(r, single, synth.bbox_diag(X), "batched vs one call per pair, g = s")
