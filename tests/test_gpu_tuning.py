"""Every force-kernel tile shape the autotuner can pick gives oracle-parity
forces, tuning in place keeps descriptors and pose, and the autotuner's
cache round-trips."""
import numpy as np
import pytest

import oracle as O
from paper_1902_01061_gb300 import autotune, scgr, synth
from tests.gpu_helpers import Gpu, check, check_pose, check_rows, rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib(scgr_lib):
    return scgr_lib


@pytest.mark.parametrize("P,tpb,splits,occ", [(1, 128, 0, 0), (2, 128, 0, 0), (4, 128, 0, 0), (1, 256, 0, 0),
                                              (2, 256, 0, 0), (4, 256, 0, 0), (4, 256, 1, 0), (2, 128, 7, 0),
                                              (1, 128, 0, 1), (2, 128, 0, 1), (4, 128, 0, 1), (1, 256, 0, 1),
                                              (2, 256, 0, 1), (4, 128, 0, 2), (2, 256, 0, 2), (4, 128, 3, 2),
                                              (2, 256, 5, 2)])
def test_every_tile_shape_matches_oracle(P, tpb, splits, occ):
    sc = synth.scale_case()
    X = sc.X[synth.subsample(sc.X, 2600, 61)]
    Y0 = sc.Y0[synth.subsample(sc.Y0, 1777, 62)]
    d = O.descriptors(X, Y0, O.Params(p=2.0))
    f_ref, W_ref = O.forces(Y0, X, d["aY"], d["aX"], d["sigma"], 2.0, 1)
    with Gpu(X, Y0, p=2.0) as g:
        scgr.scgr_set_tuning(g.ctx, scgr.SCGR_TUNE_FORCE_P, P)
        scgr.scgr_set_tuning(g.ctx, scgr.SCGR_TUNE_FORCE_TPB, tpb)
        scgr.scgr_set_tuning(g.ctx, scgr.SCGR_TUNE_FORCE_SPLITS, splits)
        scgr.scgr_set_tuning(g.ctx, scgr.SCGR_TUNE_FORCE_OCC, occ)
        plan = scgr.scgr_get_plan(g.ctx)
        assert (plan["P"], plan["tpb"], plan["occ"]) == (P, tpb, occ)
        if splits:
            # tiles are dealt in equal runs, so the count can come out below the request
            assert 1 <= plan["splits"] <= splits
        f4 = g.forces()
    check(f"force f_i, tile shape P={P} tpb={tpb} splits={splits} occ={occ}: relative L2", rel_l2(f4[:, :3], f_ref), 1e-5)
    check(f"weight W_i, tile shape P={P} tpb={tpb} splits={splits} occ={occ}: relative L2", rel_l2(f4[:, 3], W_ref), 1e-5)
    check_rows(f"force rows, tile shape P={P} tpb={tpb} splits={splits} occ={occ}", f4, f_ref, W_ref, Y0, X,
               d["aY"], d["aX"], d["sigma"], 2.0, 1)


@pytest.mark.parametrize("P,tpb", [(1, 128), (2, 256), (4, 256)])
def test_rsqrt_distance_form_matches_oracle(P, tpb):
    """p = 2 with d = d^2 rsqrt(d^2): same parity bar.  The template holds
    exact copies of reference points (d^2 = 0 pairs), which must give weight
    0, not NaN."""
    sc = synth.scale_case()
    X = sc.X[synth.subsample(sc.X, 2600, 63)]
    Y0 = np.concatenate([sc.Y0[synth.subsample(sc.Y0, 1500, 64)], X[:300]])
    d = O.descriptors(X, Y0, O.Params(p=2.0))
    f_ref, W_ref = O.forces(Y0, X, d["aY"], d["aX"], d["sigma"], 2.0, 1)
    with Gpu(X, Y0, p=2.0) as g:
        scgr.scgr_set_tuning(g.ctx, scgr.SCGR_TUNE_FORCE_P, P)
        scgr.scgr_set_tuning(g.ctx, scgr.SCGR_TUNE_FORCE_TPB, tpb)
        scgr.scgr_set_tuning(g.ctx, scgr.SCGR_TUNE_FORCE_RSQRT, 1)
        f_rs = g.forces()
        scgr.scgr_set_tuning(g.ctx, scgr.SCGR_TUNE_FORCE_RSQRT, 2)
        f_sq = g.forces()
        with pytest.raises(scgr.ScgrError):
            scgr.scgr_set_tuning(g.ctx, scgr.SCGR_TUNE_FORCE_RSQRT, 3)
    assert np.isfinite(f_rs).all()
    check("force f_i, rsqrt distance form: relative L2", rel_l2(f_rs[:, :3], f_ref), 1e-5)
    check("weight W_i, rsqrt distance form: relative L2", rel_l2(f_rs[:, 3], W_ref), 1e-5)
    check("rsqrt vs sqrt distance form: relative L2", rel_l2(f_rs, f_sq), 1e-5)
    for what, f4 in (("rsqrt", f_rs), ("sqrt", f_sq)):
        check_rows(f"force rows, {what} distance form (template holds copies of reference points)", f4, f_ref, W_ref,
                   Y0, X, d["aY"], d["aX"], d["sigma"], 2.0, 1)


@pytest.mark.parametrize("P,tpb,exo", [(4, 128, 1), (4, 128, 2), (2, 256, 1), (2, 256, 2)])
def test_fp32_pipe_exponential_matches_oracle(P, tpb, exo):
    """p = 2 with part of the similarity exponentials evaluated on the FP32
    pipe (SCGR_TUNE_FORCE_EX2POLY) in the shared-memory-sum shapes: the same
    parity bar, per row as well.  The template holds exact copies of
    reference points (d = 0 pairs) and the padding of the last tiles has
    infinite exponents, which must give weight 0."""
    sc = synth.scale_case()
    X = sc.X[synth.subsample(sc.X, 2600, 65)]
    Y0 = np.concatenate([sc.Y0[synth.subsample(sc.Y0, 1500, 66)], X[:300]])
    d = O.descriptors(X, Y0, O.Params(p=2.0))
    f_ref, W_ref = O.forces(Y0, X, d["aY"], d["aX"], d["sigma"], 2.0, 1)
    with Gpu(X, Y0, p=2.0) as g:
        scgr.scgr_set_tuning(g.ctx, scgr.SCGR_TUNE_FORCE_P, P)
        scgr.scgr_set_tuning(g.ctx, scgr.SCGR_TUNE_FORCE_TPB, tpb)
        scgr.scgr_set_tuning(g.ctx, scgr.SCGR_TUNE_FORCE_OCC, 2)
        scgr.scgr_set_tuning(g.ctx, scgr.SCGR_TUNE_FORCE_EX2POLY, exo)
        plan = scgr.scgr_get_plan(g.ctx)
        assert (plan["P"], plan["tpb"], plan["occ"]) == (P, tpb, 2)
        f_poly = g.forces()
        scgr.scgr_set_tuning(g.ctx, scgr.SCGR_TUNE_FORCE_EX2POLY, 0)
        f_mufu = g.forces()
        with pytest.raises(scgr.ScgrError):
            scgr.scgr_set_tuning(g.ctx, scgr.SCGR_TUNE_FORCE_EX2POLY, 3)
    assert np.isfinite(f_poly).all()
    what = f"FP32-pipe exponential, P={P} tpb={tpb}, {exo} of {2 * P} pair updates per step"
    check(f"force f_i, {what}: relative L2", rel_l2(f_poly[:, :3], f_ref), 1e-5)
    check(f"weight W_i, {what}: relative L2", rel_l2(f_poly[:, 3], W_ref), 1e-5)
    check(f"{what} vs special-function ex2: relative L2", rel_l2(f_poly, f_mufu), 1e-5)
    check_rows(f"force rows, {what}", f_poly, f_ref, W_ref, Y0, X, d["aY"], d["aX"], d["sigma"], 2.0, 1)


def test_autotuner_picks_and_caches(tmp_path, monkeypatch):
    monkeypatch.setenv("SCGR_TUNE_CACHE", str(tmp_path / "tune.json"))
    case = synth.mild(n=3000)
    with Gpu(case.X, case.Y0, p=2.0) as g:
        best = autotune.tune_single(g.ctx, len(case.X), len(case.Y0), 2.0,
                                    candidates=[(1, 128, 0), (2, 256, 1)], reps=2)
        plan = scgr.scgr_get_plan(g.ctx)
        assert (plan["P"], plan["tpb"]) == (best["P"], best["tpb"])
        assert len(best["tried"]) == 4 and best["ms"] > 0          # two shapes, then both again in rsqrt form
    with Gpu(case.X, case.Y0, p=2.0) as g:
        hit = autotune.apply_cached_single(g.ctx, len(case.X), len(case.Y0), 2.0)
        assert hit is not None and hit["P"] == best["P"]
        plan = scgr.scgr_get_plan(g.ctx)
        assert (plan["P"], plan["tpb"]) == (best["P"], best["tpb"])


@pytest.mark.parametrize("use_graph", [0, 1])
def test_p1_force_sums_reused_bit_identically(use_graph):
    """p = 1: the pose-free force sums computed once per run give the same
    bits as recomputing them every iteration, with fewer launches."""
    case = synth.mild(n=1200)
    with Gpu(case.X, case.Y0, p=1.0, use_graph=use_graph) as g:
        a = g.run(30)
        na = scgr.scgr_launch_count(g.ctx)
    with Gpu(case.X, case.Y0, p=1.0, use_graph=use_graph) as g:
        scgr.scgr_set_tuning(g.ctx, scgr.SCGR_TUNE_REUSE_POSE_FREE, 0)
        b = g.run(30)
        nb = scgr.scgr_launch_count(g.ctx)
    assert list(a.R) == list(b.R) and list(a.t) == list(b.t) and a.s == b.s
    assert nb - na == 29


def test_p3_moment_path_matches_all_pairs_and_oracle():
    """p = 3: 14 pose-free moments once per run instead of an all-pairs pass
    per iteration; equal to the all-pairs path (and the oracle) within the
    pose tolerance."""
    case = synth.mild(n=1500)
    iters = 25
    with Gpu(case.X, case.Y0, p=3.0) as g:
        scgr.scgr_set_force_timing(g.ctx, True)
        a = g.run(iters)
        na = scgr.scgr_get_force_timing(g.ctx)[0]
    with Gpu(case.X, case.Y0, p=3.0) as g:
        scgr.scgr_set_tuning(g.ctx, scgr.SCGR_TUNE_REUSE_POSE_FREE, 0)
        scgr.scgr_set_force_timing(g.ctx, True)
        b = g.run(iters)
        nb = scgr.scgr_get_force_timing(g.ctx)[0]
    o = O.register(case.X, case.Y0, O.Params(p=3.0), iterations=iters)
    diag = synth.bbox_diag(case.X)
    for what, r in (("pose, p = 3 moment path", a), ("pose, p = 3 all-pairs path", b)):
        R, t, s = r.as_numpy()
        check_pose(what, R, t, s, o["R"], o["t"], o["s"], diag)
    assert (na, nb) == (0, iters)        # one moments pass replaces the 25 all-pairs force launches


def test_small_problem_splits_reference_down_to_half_tiles():
    """A problem whose one-tile-per-block grid fills less than half a wave
    (the 1,000-point case: 8 template blocks, 4 tiles) splits every
    reference tile in two (8 splits of 128 points), and the forces keep
    oracle parity."""
    case = synth.tiny()
    d = O.descriptors(case.X, case.Y0, O.Params(p=2.0))
    f_ref, W_ref = O.forces(case.Y0, case.X, d["aY"], d["aX"], d["sigma"], 2.0, 1)
    with Gpu(case.X, case.Y0, p=2.0) as g:
        plan = scgr.scgr_get_plan(g.ctx)
        assert plan["splits"] == 8 and plan["iblocks"] == 8, plan
        f4 = g.forces()
    check("force f_i, 1000 x 1000 with half a tile per split: relative L2", rel_l2(f4[:, :3], f_ref), 1e-5)
    check_rows("force rows, 1000 x 1000 with half a tile per split", f4, f_ref, W_ref, case.Y0, case.X,
               d["aY"], d["aX"], d["sigma"], 2.0, 1)
