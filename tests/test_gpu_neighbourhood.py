"""Neighbourhood variants on the GPU against the oracle: the radius
neighbourhood of Sec. IV (radius sqrt(e) times a scale) and the pyramidal
schedule (neighbourhood and sigma shrinking between levels, pose kept)."""
import numpy as np
import pytest

import oracle as O
from paper_1902_01061_gb300 import scgr, synth
from tests.gpu_helpers import Gpu, check, check_pose

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib(scgr_lib):
    return scgr_lib


def pose_close(res, o, diag, what):
    R, t, s = res.as_numpy()
    check_pose(what, R, t, s, o["R"], o["t"], o["s"], diag)
    return True


@pytest.mark.parametrize("scale", [1.0, 0.35])
def test_radius_curvature_matches_oracle(scale):
    case = synth.mild(n=1500)
    with Gpu(case.X, case.Y0, neigh_mode=1, radius_scale=scale) as g:
        for which, P in ((0, case.X), (1, case.Y0)):
            a_ref = O.curvature_radius(P, scale)
            a_got = g.curv64(which)
            np.testing.assert_allclose(a_got, a_ref, rtol=1e-5, atol=1e-10)
            check("radius curvature: max |da| / (|a| + 1e-5)", np.max(np.abs(a_got - a_ref) / (np.abs(a_ref) + 1e-5)),
                  1e-5)
        assert g.sigma() == pytest.approx(O.sigma_auto(O.curvature_radius(case.X, scale)), rel=1e-5)


def test_radius_mode_registration_matches_oracle():
    case = synth.mild(n=800)
    prm = O.Params(neigh_mode=1, radius_scale=0.4)
    o = O.register(case.X, case.Y0, prm, iterations=20)
    with Gpu(case.X, case.Y0, neigh_mode=1, radius_scale=0.4) as g:
        assert pose_close(g.run(20), o, synth.bbox_diag(case.X), "pose, radius neighbourhood")


@pytest.mark.parametrize("mode", [0, 1])
def test_pyramid_matches_oracle(mode):
    case = synth.mild(n=900)
    if mode == 0:
        levels = [(10, 24, 1.0, 1.5), (10, 16, 1.0, 1.0), (10, 8, 1.0, 0.7)]
    else:
        levels = [(10, 16, 0.6, 1.5), (10, 16, 0.4, 1.0), (10, 16, 0.25, 0.7)]
    prm = O.Params(neigh_mode=mode)
    o = O.register_pyramid(case.X, case.Y0, prm, levels)
    with Gpu(case.X, case.Y0, neigh_mode=mode, E=30) as g:
        res = scgr.run_pyramid(g.ctx, levels)
    assert res.iterations == 30
    assert pose_close(res, o, synth.bbox_diag(case.X), f"pose, pyramidal schedule (mode {mode})")


def test_set_neighbourhood_rejects_bad_values():
    case = synth.mild(n=300)
    with Gpu(case.X, case.Y0) as g:
        for args in ((2, 1.0, 1.0), (33, 1.0, 1.0), (16, 0.0, 1.0), (16, 1.0, -1.0)):
            with pytest.raises(scgr.ScgrError):
                scgr.scgr_set_neighbourhood(g.ctx, *args)


@pytest.mark.parametrize("grid", [False, True])
def test_nearest_bit_exact(grid):
    """Brute force and (forced) exact grid search against the oracle, with
    queries inside and far outside the reference's box, queries on reference
    points, and duplicated reference points (ties to the lower index)."""
    import torch
    sc = synth.scale_case()
    X = sc.X[synth.subsample(sc.X, 3000, 71)]
    X = np.concatenate([X, X[:50]])                  # exact duplicates: equal keys
    Q = sc.Y0[synth.subsample(sc.Y0, 1200, 72)]
    far = (3.0 * Q[:100] + np.float32(2.5)).astype(np.float32)
    Q = np.concatenate([Q, far, X[:40], X[3000:3010]]).astype(np.float32)
    idx_ref, key_ref = O.nearest(Q, X)
    tune = {scgr.SCGR_TUNE_NEAREST_GRID_MIN: 0 if grid else 1 << 30}
    with Gpu(X, X, tune=tune) as g:
        idx = torch.empty(len(Q), dtype=torch.int32, device="cuda")
        key = torch.empty(len(Q), dtype=torch.float32, device="cuda")
        scgr.scgr_nearest(g.ctx, torch.from_numpy(Q).cuda(), idx, key)
        np.testing.assert_array_equal(idx.cpu().numpy(), idx_ref)
        np.testing.assert_array_equal(key.cpu().numpy(), key_ref)


def test_nearest_grid_at_full_size():
    """The 1M-point reference of the benchmark workload (grid search by
    default): 4,096 template points and 512 points outside the box, equal to
    the brute-force kernel on every query and to the oracle on sampled ones."""
    import torch
    big = synth.large_case()
    rng = np.random.default_rng(83)
    Q = big.Y0[rng.choice(len(big.Y0), size=4096, replace=False)]
    Q = np.concatenate([Q, (Q[:512] * 2.0 + np.float32(1.5)).astype(np.float32)])
    Qd = torch.from_numpy(Q).cuda()
    out = {}
    for name, gmin in (("grid", 65536), ("brute", 1 << 30)):
        with Gpu(big.X, big.Y0[:64], tune={scgr.SCGR_TUNE_NEAREST_GRID_MIN: gmin}) as g:
            idx = torch.empty(len(Q), dtype=torch.int32, device="cuda")
            key = torch.empty(len(Q), dtype=torch.float32, device="cuda")
            scgr.scgr_nearest(g.ctx, Qd, idx, key)
            out[name] = (idx.cpu().numpy(), key.cpu().numpy())
    check("nearest: grid vs brute-force indices differing (1M reference)",
          np.count_nonzero(out["grid"][0] != out["brute"][0]), 0)
    np.testing.assert_array_equal(out["grid"][1], out["brute"][1])
    sample = np.concatenate([np.arange(0, 4096, 97), np.arange(4096, 4608, 31)])
    idx_ref, key_ref = O.nearest(Q[sample], big.X)
    check("nearest: grid vs oracle indices differing (1M reference, sampled queries)",
          np.count_nonzero(out["grid"][0][sample] != idx_ref), 0)
    np.testing.assert_array_equal(out["grid"][1][sample], key_ref)


def test_nearest_two_level_search_off_surface_queries():
    """The two-level search (fine cells, then coarse cells skipping empty
    space) and the fine-shell search give the same (key, index)-first point
    as the brute force for queries spread through the 1M reference's box,
    most of them off the surface, plus queries on reference points and far
    outside the box; the second query pass reuses the cached grids."""
    import torch
    big = synth.large_case()
    rng = np.random.default_rng(91)
    lo, hi = big.X.min(axis=0), big.X.max(axis=0)
    Q = np.concatenate([rng.uniform(lo, hi, size=(3000, 3)).astype(np.float32),
                        big.X[rng.choice(len(big.X), size=500, replace=False)],
                        (hi + np.float32(1.0) + rng.uniform(0, 2, size=(200, 3))).astype(np.float32)])
    Qd = torch.from_numpy(Q).cuda()
    out = {}
    for name, gmin, levels in (("two-level", 65536, 2), ("fine", 65536, 1), ("brute", 1 << 30, 2)):
        with Gpu(big.X, big.Y0[:64], tune={scgr.SCGR_TUNE_NEAREST_GRID_MIN: gmin,
                                           scgr.SCGR_TUNE_NEAREST_LEVELS: levels}) as g:
            idx = torch.empty(len(Q), dtype=torch.int32, device="cuda")
            key = torch.empty(len(Q), dtype=torch.float32, device="cuda")
            for _ in range(2):
                scgr.scgr_nearest(g.ctx, Qd, idx, key)
            out[name] = (idx.cpu().numpy(), key.cpu().numpy())
    for name in ("two-level", "fine"):
        check(f"nearest: {name} grid search vs brute force, indices differing (1M reference, off-surface queries)",
              np.count_nonzero(out[name][0] != out["brute"][0]), 0)
        np.testing.assert_array_equal(out[name][1], out["brute"][1])


@pytest.mark.parametrize("grid", [False, True])
def test_change_mask_at_identity_pose(grid):
    """A template whose part moved between captures: the moved part is
    flagged.  At the identity pose the moved template is Y0 itself, so the
    oracle gets exactly the GPU's query points."""
    import torch
    rng = np.random.default_rng(81)
    surf = synth.EllipsoidUnion.random(rng, 3)
    X = surf.sample_surface(rng, 2000).astype(np.float32)
    Y0 = X[synth.subsample(X, 1500, 82)].copy()
    Y0[:200] += np.float32(0.2)                      # a part that moved
    thr = 0.05
    mask_ref, dist_ref = O.change_mask(Y0, X, thr)
    with Gpu(X, Y0, tune={scgr.SCGR_TUNE_NEAREST_GRID_MIN: 0 if grid else 1 << 30}) as g:
        mask = torch.empty(len(Y0), dtype=torch.uint8, device="cuda")
        dist = torch.empty(len(Y0), dtype=torch.float32, device="cuda")
        scgr.scgr_change_mask(g.ctx, thr, mask, dist)
        np.testing.assert_array_equal(mask.cpu().numpy(), mask_ref)
        np.testing.assert_allclose(dist.cpu().numpy(), dist_ref, rtol=1e-6)
    assert mask_ref[:200].mean() > 0.5 and mask_ref[200:].mean() < 0.05


def test_nearest_two_level_search_on_degenerate_references():
    """The two-level nearest search over references whose grids collapse to
    one cell along some axes (a plane, a line, coincident points), with
    queries on, near and far from them: equal to the oracle."""
    import torch
    rng = np.random.default_rng(93)
    plane = np.c_[rng.uniform(-1, 1, (3000, 2)), np.zeros(3000)].astype(np.float32)
    line = np.c_[np.linspace(0, 1, 1500), np.linspace(0, 2, 1500), np.zeros(1500)].astype(np.float32)
    same = np.tile(np.array([[0.5, -0.25, 2.0]], np.float32), (64, 1))
    for X in (plane, line, same):
        Q = np.concatenate([X[rng.choice(len(X), 200)],
                            (X[rng.choice(len(X), 200)] + rng.normal(0, 0.05, (200, 3))).astype(np.float32),
                            rng.uniform(-3, 3, (200, 3)).astype(np.float32)])
        idx_ref, key_ref = O.nearest(Q, X)
        with Gpu(X, X, tune={scgr.SCGR_TUNE_NEAREST_GRID_MIN: 0}) as g:
            idx = torch.empty(len(Q), dtype=torch.int32, device="cuda")
            key = torch.empty(len(Q), dtype=torch.float32, device="cuda")
            scgr.scgr_nearest(g.ctx, torch.from_numpy(Q).cuda(), idx, key)
            check("nearest, degenerate reference: indices differing from the oracle",
                  np.count_nonzero(idx.cpu().numpy() != idx_ref), 0)
            np.testing.assert_array_equal(key.cpu().numpy(), key_ref)
