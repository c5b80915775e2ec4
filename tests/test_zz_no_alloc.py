"""scgr_forces_static, the force entry point for callers that cannot allocate
device memory (their memory belongs to another allocator, or a real-time loop
cannot take cudaMalloc/cudaFree), must give the same forces as the context
path (scgr_forces after scgr_set_curvature) within the force tolerance of the
other tests.  It keeps all scratch in one static device array shared by every
call, so calls in a row with different inputs must not see each other's
leftovers: a small call after a larger one repeats an earlier small call bit
for bit, leaves the device's free memory unchanged, and a good call after a
rejected one succeeds.  This file is collected last on purpose."""
import numpy as np
import pytest
import torch

from paper_1902_01061_gb300 import scgr, synth
from tests.gpu_helpers import Gpu, rel_l2

pytestmark = pytest.mark.gpu

FORCE_TOL = 1e-5


def curvatures(n, seed):
    rng = np.random.default_rng(seed)
    return np.clip(rng.gamma(1.2, 0.015, size=n), 0.0, 0.33)


def context_forces(X, Y0, aX, aY, p):
    with Gpu(X, Y0, p=p) as g:
        g.set_curvature(0, aX)
        g.set_curvature(1, aY)
        return g.forces()


def static_forces(X, Y0, aX, aY, p):
    out = torch.full((len(Y0), 4), float("nan"), dtype=torch.float32, device="cuda")
    scgr.scgr_forces_static(torch.from_numpy(X).cuda(), torch.from_numpy(Y0).cuda(),
                            torch.from_numpy(aX).cuda(), torch.from_numpy(aY).cuda(), out, p=p, g_mode=1)
    return out.cpu().numpy()


def test_static_forces_match_context_path_two_calls_in_a_row(scgr_lib):
    a = synth.mild(n=1000)
    sc = synth.scale_case()
    Xb = sc.X[synth.subsample(sc.X, 5000, 31)]
    Yb = sc.Y0[synth.subsample(sc.Y0, 3001, 32)]
    cases = [(a.X, a.Y0, curvatures(1000, 1), curvatures(1000, 2), 2.0),
             (Xb, Yb, curvatures(5000, 3), curvatures(3001, 4), 1.5)]
    outs = []
    for X, Y0, aX, aY, p in cases:          # two calls in a row, different sizes
        want = context_forces(X, Y0, aX, aY, p)
        got = static_forces(X, Y0, aX, aY, p)
        assert np.isfinite(got).all()
        assert rel_l2(got[:, :3], want[:, :3]) <= FORCE_TOL
        assert rel_l2(got[:, 3], want[:, 3]) <= FORCE_TOL
        outs.append(got)
    # back to the small case after the larger one: leftovers of the larger
    # call in the shared array (padded records, partial sums, the error word)
    # must not reach the result, which repeats the first call bit for bit
    X, Y0, aX, aY, p = cases[0]
    dev = [torch.from_numpy(v).cuda() for v in (X, Y0, aX, aY)]
    out = torch.full((len(Y0), 4), float("nan"), dtype=torch.float32, device="cuda")
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    scgr.scgr_forces_static(*dev, out, p=p, g_mode=1)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0          # the call holds no device memory of its own
    np.testing.assert_array_equal(out.cpu().numpy(), outs[0])


def test_good_call_after_a_rejected_one(scgr_lib):
    """A call whose input sets the device error word (a curvature outside
    [0, 1]) returns SCGR_ERR_NONFINITE; the next good call starts from a
    cleared error word and returns the forces of a fresh call."""
    a = synth.mild(n=700)
    aX, aY = curvatures(700, 5), curvatures(700, 6)
    first = static_forces(a.X, a.Y0, aX, aY, 2.0)
    bad = aX.copy()
    bad[3] = 2.0
    with pytest.raises(scgr.ScgrError) as e:
        static_forces(a.X, a.Y0, bad, aY, 2.0)
    assert e.value.status == 3
    np.testing.assert_array_equal(static_forces(a.X, a.Y0, aX, aY, 2.0), first)


def test_static_forces_reject_oversize_and_bad_input(scgr_lib):
    big = torch.zeros((131073, 3), dtype=torch.float32, device="cuda")
    a = torch.zeros(131073, dtype=torch.float64, device="cuda")
    out = torch.empty((16, 4), dtype=torch.float32, device="cuda")
    small = torch.zeros((16, 3), dtype=torch.float32, device="cuda")
    with pytest.raises(scgr.ScgrError) as e:
        scgr.scgr_forces_static(big, small, a, a[:16], out)
    assert e.value.status == 1
    bad = torch.full((16,), 2.0, dtype=torch.float64, device="cuda")     # curvature outside [0, 1]
    with pytest.raises(scgr.ScgrError) as e:
        scgr.scgr_forces_static(small + torch.arange(16, device="cuda")[:, None].float(), small,
                                bad, a[:16], out)
    assert e.value.status == 3
