"""Differentiation form on the GPU: the potential U and its hand-written
adjoint (pose gradient in axis-angle, t, s and template-coordinate gradient)
against the FP64 oracle's analytic gradient and against central finite
differences (h = 1e-4) of the oracle's FP64 potential (descriptors fixed).
Bar: gradients within 1e-4 relative; U within 1e-6 relative."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_1902_01061_gb300 import scgr, synth
from tests.gpu_helpers import Gpu, check, rel_l2

pytestmark = pytest.mark.gpu

POSES = [np.array([0.3, -0.2, 0.5, 0.1, 0.2, -0.3, 1.2]),
         np.array([0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 1.0]),
         np.array([-1.1, 0.4, 2.0, -0.05, 0.0, 0.4, 0.8])]


@pytest.fixture(scope="module", autouse=True)
def _lib(scgr_lib):
    return scgr_lib


def curvatures(n, seed):
    rng = np.random.default_rng(seed)
    return np.clip(rng.gamma(1.2, 0.015, size=n), 0.0, 0.33)


def block_rel(a, b):
    """relative errors of the (omega, t, s) blocks of a pose gradient"""
    return [rel_l2(a[sl], b[sl]) for sl in (slice(0, 3), slice(3, 6), slice(6, 7))]


@pytest.mark.parametrize("p", [1.0, 2.0, 1.5])
def test_potential_and_adjoint_match_oracle_analytic(p):
    case = synth.mild(n=900)
    d = O.descriptors(case.X, case.Y0, O.Params(p=p))
    with Gpu(case.X, case.Y0, p=p) as g:
        for pose in POSES:
            gx = torch.empty((g.m, 3), dtype=torch.float32, device="cuda")
            U, g7 = scgr.scgr_potential(g.ctx, pose, want_grad=True, grad_xyz_out=gx)
            Uo, g7o, gY0o = O.pose_potential_and_grad(pose, case.Y0, case.X, d["aY"], d["aX"], d["sigma"], p, 1)
            check(f"potential U (p={p:g}): relative error", abs(U - Uo) / abs(Uo), 1e-6)
            check(f"pose gradient (p={p:g}) vs oracle: worst block relative L2", max(block_rel(g7, g7o)), 1e-4)
            check(f"template-point gradient (p={p:g}) vs oracle: relative L2", rel_l2(gx.cpu().numpy(), gY0o), 1e-5)
            U2, none = scgr.scgr_potential(g.ctx, pose, want_grad=False)
            assert U2 == U and none is None


def test_adjoint_matches_central_differences_of_oracle_potential():
    """Config-3 shaped input (rotation 30 deg, noise 0.01 of the diagonal),
    subsampled so that 14 oracle potentials finish in seconds."""
    dc = synth.diff_case(n=50_000)
    X = dc.X[synth.subsample(dc.X, 1500, 41)]
    Y0 = dc.Y0[synth.subsample(dc.Y0, 1400, 42)]
    p = 2.0
    d = O.descriptors(X, Y0, O.Params(p=p))
    pose = np.array([0.2, 0.1, -0.3, 0.05, -0.1, 0.02, 1.05])
    h = 1e-4
    fd = np.zeros(7)
    for q in range(7):
        pp = pose.copy(); pp[q] += h
        pm = pose.copy(); pm[q] -= h
        Up = O.pose_potential_and_grad(pp, Y0, X, d["aY"], d["aX"], d["sigma"], p, 1)[0]
        Um = O.pose_potential_and_grad(pm, Y0, X, d["aY"], d["aX"], d["sigma"], p, 1)[0]
        fd[q] = (Up - Um) / (2 * h)
    with Gpu(X, Y0, p=p) as g:
        _, g7 = scgr.scgr_potential(g.ctx, pose)
    check("pose gradient vs central differences (h = 1e-4): worst block relative L2", max(block_rel(g7, fd)), 1e-4)


def test_autograd_function_backward():
    case = synth.mild(n=700)
    p = 2.0
    d = O.descriptors(case.X, case.Y0, O.Params(p=p))
    with Gpu(case.X, case.Y0, p=p) as g:
        pose = torch.tensor(POSES[0], dtype=torch.float64, requires_grad=True)
        Y0 = g.Y0.clone().requires_grad_(True)
        U = scgr.potential(pose, Y0, g.ctx)
        (3.0 * U).backward()
        Uo, g7o, gY0o = O.pose_potential_and_grad(POSES[0], case.Y0, case.X, d["aY"], d["aX"], d["sigma"], p, 1)
        check("autograd potential: relative error", abs(U.item() - Uo) / abs(Uo), 1e-6)
        check("autograd pose gradient: worst block relative L2", max(block_rel(pose.grad.numpy(), 3.0 * g7o)), 1e-4)
        check("autograd template-point gradient: relative L2", rel_l2(Y0.grad.cpu().numpy(), 3.0 * gY0o), 1e-5)


def test_full_size_50k_sampled_rows_and_identities():
    """50,000 x 50,000 (config 3): per-point gradients at sampled rows against
    the oracle (seeded descriptors on both sides), dU/dt = -F (total force from
    scgr_forces at the same pose), and U against the force kernel's W sums."""
    dc = synth.diff_case()
    rng = np.random.default_rng(3)
    aX = curvatures(len(dc.X), 51)
    aY = curvatures(len(dc.Y0), 52)
    sigma = O.sigma_auto(aX)
    p = 2.0
    pose = np.array([0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 1.0])   # identity: scgr_forces evaluates here too
    with Gpu(dc.X, dc.Y0, p=p) as g:
        g.set_curvature(0, aX)
        g.set_curvature(1, aY)
        gx = torch.empty((g.m, 3), dtype=torch.float32, device="cuda")
        U, g7 = scgr.scgr_potential(g.ctx, pose, grad_xyz_out=gx)
        f4 = g.forces()
    rows = np.sort(rng.choice(len(dc.Y0), size=64, replace=False))
    fr, _ = O.forces_rows(dc.Y0, dc.X, aY, aX, sigma, p, 1, rows)
    check("template-point gradient, 50k x 50k sampled rows: relative L2", rel_l2(gx.cpu().numpy()[rows], -fr), 1e-5)
    F = f4[:, :3].astype(np.float64).sum(axis=0)
    check("dU/dt + F, 50k x 50k: relative L2", rel_l2(g7[3:6], -F), 1e-5)
    assert U > 0 and np.isfinite(g7).all()


@pytest.mark.parametrize("p", [1.0, 2.0, 1.5])
def test_force_vjp_matches_oracle(p):
    case = synth.mild(n=700)
    d = O.descriptors(case.X, case.Y0, O.Params(p=p))
    v = np.random.default_rng(4).normal(size=(len(case.Y0), 3)).astype(np.float32)
    ref = O.force_vjp(case.Y0, case.X, d["aY"], d["aX"], d["sigma"], p, 1, v)
    with Gpu(case.X, case.Y0, p=p) as g:
        out = torch.empty((g.m, 3), dtype=torch.float32, device="cuda")
        scgr.scgr_force_vjp(g.ctx, torch.from_numpy(v).cuda(), out)
        got = out.cpu().numpy()
    check(f"force VJP (p={p:g}) vs oracle: relative L2", rel_l2(got, ref), 1e-5)


@pytest.mark.parametrize("p", [2.0, 1.0])
def test_stored_pair_terms_match_recomputation(p):
    case = synth.mild(n=800)
    d = O.descriptors(case.X, case.Y0, O.Params(p=p))
    pose = POSES[0]
    with Gpu(case.X, case.Y0, p=p) as g:
        gx_r = torch.empty((g.m, 3), dtype=torch.float32, device="cuda")
        gx_s = torch.empty((g.m, 3), dtype=torch.float32, device="cuda")
        U_r, g_r = scgr.scgr_potential(g.ctx, pose, grad_xyz_out=gx_r)
        U_s, g_s = scgr.scgr_potential_stored(g.ctx, pose, grad_xyz_out=gx_s)
    Uo, g7o, gY0o = O.pose_potential_and_grad(pose, case.Y0, case.X, d["aY"], d["aX"], d["sigma"], p, 1)
    check(f"potential, stored pair terms (p={p:g}): relative error", abs(U_s - Uo) / abs(Uo), 1e-6)
    check(f"potential, recomputed tiles (p={p:g}): relative error", abs(U_r - Uo) / abs(Uo), 1e-6)
    check(f"pose gradient, stored pair terms (p={p:g}): worst block relative L2", max(block_rel(g_s, g7o)), 1e-4)
    check(f"pose gradient, recomputed tiles (p={p:g}): worst block relative L2", max(block_rel(g_r, g7o)), 1e-4)
    check(f"template-point gradient, stored pair terms (p={p:g}): relative L2",
          rel_l2(gx_s.cpu().numpy(), gY0o), 1e-5)
