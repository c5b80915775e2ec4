"""Thin ctypes binding of libscgr.so (include/scgr.h).

Argument marshalling only: every step of the method runs in the CUDA
library.  Functions keep the C names; device arrays are torch CUDA tensors
(float32 [n, 3] contiguous for clouds), host arrays are numpy arrays.  There
is no CPU fallback: if the library is not built, the first call raises.
"""
from __future__ import annotations

import ctypes
import os
from ctypes import POINTER, Structure, c_char_p, c_double, c_float, c_int, c_int32, c_int64, c_void_p

import numpy as np

LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libscgr.so")

SCGR_OK = 0
STATUS_NAMES = {
    0: "SCGR_OK", 1: "SCGR_ERR_INVALID_ARG", 2: "SCGR_ERR_STATE", 3: "SCGR_ERR_NONFINITE",
    4: "SCGR_ERR_OOM", 5: "SCGR_ERR_CUDA", 6: "SCGR_ERR_TIMEOUT", 7: "SCGR_ERR_NUMERIC",
}

# every symbol include/scgr.h declares (checked by the CPU test-suite)
EXPORTED = (
    "scgr_default_params", "scgr_create", "scgr_destroy", "scgr_last_error",
    "scgr_set_reference", "scgr_set_reference_host", "scgr_set_template", "scgr_set_template_host",
    "scgr_compute_descriptors", "scgr_run", "scgr_get_result", "scgr_get_moved",
    "scgr_get_moved_host", "scgr_get_descriptors", "scgr_get_sigma", "scgr_get_curvature64",
    "scgr_forces", "scgr_get_state", "scgr_set_state", "scgr_sync", "scgr_launch_count",
    "scgr_set_curvature", "scgr_set_force_timing", "scgr_get_force_timing", "scgr_forces_static",
    "scgr_potential", "scgr_batch_run", "scgr_set_tuning", "scgr_set_row_range", "scgr_step_partials",
    "scgr_step_apply", "scgr_get_plan", "scgr_microbench", "scgr_set_neighbourhood", "scgr_nearest",
    "scgr_change_mask", "scgr_force_vjp", "scgr_potential_stored", "scgr_debug_fail_allocations",
    "scgr_step_partials_dev", "scgr_step_apply_dev", "scgr_plan_preview",
)
SCGR_TUNE_BATCH_CHUNK_TILES = 1
SCGR_TUNE_KNN_GRID_MIN = 2
SCGR_TUNE_FORCE_P = 3
SCGR_TUNE_FORCE_TPB = 4
SCGR_TUNE_FORCE_SPLITS = 5
SCGR_TUNE_REUSE_POSE_FREE = 6
SCGR_TUNE_FORCE_OCC = 7
SCGR_TUNE_BATCH_P = 8
SCGR_TUNE_BATCH_PERSISTENT = 10
SCGR_TUNE_FORCE_RSQRT = 9
SCGR_TUNE_FORCE_EX2POLY = 11
SCGR_TUNE_NEAREST_LEVELS = 12
SCGR_TUNE_FUSED_TAIL = 13
SCGR_TUNE_NEAREST_GRID_MIN = 14


class scgr_params(Structure):
    _fields_ = [("k", c_int), ("p", c_double), ("sigma", c_double), ("g_mode", c_int),
                ("G1", c_double), ("E", c_int), ("step_mode", c_int), ("eta0", c_double),
                ("time", c_double), ("scale_mode", c_int), ("use_graph", c_int), ("neigh_mode", c_int),
                ("radius_scale", c_double)]


class scgr_result(Structure):
    _fields_ = [("R", c_double * 9), ("t", c_double * 3), ("s", c_double),
                ("iterations", c_int), ("degenerate_steps", c_int)]

    def as_numpy(self):
        return (np.array(self.R[:]).reshape(3, 3), np.array(self.t[:]), float(self.s))


class scgr_state(Structure):
    _fields_ = [("R", c_double * 9), ("t", c_double * 3), ("s", c_double),
                ("iteration", c_int), ("E", c_int), ("degenerate_steps", c_int),
                ("sigma", c_double)]


class ScgrError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


_lib = None


def load():
    """Load libscgr.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_1902_01061_gb300.build.build()")
    L = ctypes.CDLL(LIB_PATH)
    S = c_int
    ctx = c_void_p
    sig = {
        "scgr_default_params": (S, [POINTER(scgr_params)]),
        "scgr_create": (S, [POINTER(scgr_params), c_void_p, POINTER(c_void_p)]),
        "scgr_destroy": (None, [ctx]),
        "scgr_last_error": (c_char_p, [ctx]),
        "scgr_set_reference": (S, [ctx, c_void_p, c_int64]),
        "scgr_set_reference_host": (S, [ctx, c_void_p, c_int64]),
        "scgr_set_template": (S, [ctx, c_void_p, c_int64]),
        "scgr_set_template_host": (S, [ctx, c_void_p, c_int64]),
        "scgr_compute_descriptors": (S, [ctx]),
        "scgr_run": (S, [ctx, c_int]),
        "scgr_get_result": (S, [ctx, POINTER(scgr_result)]),
        "scgr_get_moved": (S, [ctx, c_void_p]),
        "scgr_get_moved_host": (S, [ctx, c_void_p]),
        "scgr_get_descriptors": (S, [ctx, c_int, c_void_p, c_void_p]),
        "scgr_get_sigma": (S, [ctx, POINTER(c_double)]),
        "scgr_get_curvature64": (S, [ctx, c_int, c_void_p]),
        "scgr_forces": (S, [ctx, c_void_p]),
        "scgr_get_state": (S, [ctx, POINTER(scgr_state)]),
        "scgr_set_state": (S, [ctx, POINTER(scgr_state)]),
        "scgr_sync": (S, [ctx]),
        "scgr_launch_count": (c_int64, [ctx]),
        "scgr_set_curvature": (S, [ctx, c_int, c_void_p]),
        "scgr_set_force_timing": (S, [ctx, c_int]),
        "scgr_get_force_timing": (S, [ctx, POINTER(c_int64), POINTER(c_double)]),
        "scgr_batch_run": (S, [ctx, c_int, c_void_p, c_void_p, c_void_p, c_void_p, c_int, c_void_p]),
        "scgr_set_tuning": (S, [ctx, c_int, c_int]),
        "scgr_get_plan": (S, [ctx, POINTER(c_int)]),
        "scgr_set_neighbourhood": (S, [ctx, c_int, c_double, c_double]),
        "scgr_force_vjp": (S, [ctx, c_void_p, c_void_p]),
        "scgr_debug_fail_allocations": (S, [c_int]),
        "scgr_potential_stored": (S, [ctx, POINTER(c_double), POINTER(c_double), POINTER(c_double), c_void_p]),
        "scgr_nearest": (S, [ctx, c_void_p, c_int64, c_void_p, c_void_p]),
        "scgr_change_mask": (S, [ctx, c_double, c_void_p, c_void_p]),
        "scgr_microbench": (S, [c_int, c_int, c_void_p, c_void_p, POINTER(c_int64), POINTER(c_double)]),
        "scgr_set_row_range": (S, [ctx, c_int64, c_int64]),
        "scgr_step_partials": (S, [ctx, POINTER(c_double)]),
        "scgr_step_apply": (S, [ctx, POINTER(c_double)]),
        "scgr_step_partials_dev": (S, [ctx, c_void_p]),
        "scgr_step_apply_dev": (S, [ctx, c_void_p, c_int]),
        "scgr_potential": (S, [ctx, POINTER(c_double), POINTER(c_double), POINTER(c_double), c_void_p]),
        "scgr_forces_static": (S, [c_void_p, c_int64, c_void_p, c_int64, c_void_p, c_void_p, c_double,
                                   c_double, c_int, c_void_p, c_void_p]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _lib = L
    return L


def _check(status: int, ctx=None):
    if status != SCGR_OK:
        msg = load().scgr_last_error(ctx)
        raise ScgrError(status, msg.decode() if msg else "")


def _dev_ptr(t, dtype_name: str, shape_tail=None) -> int:
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError("expected a CUDA tensor")
    if str(t.dtype) != f"torch.{dtype_name}":
        raise TypeError(f"expected dtype {dtype_name}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError("tensor must be contiguous")
    if shape_tail is not None and tuple(t.shape[1:]) != tuple(shape_tail):
        raise ValueError(f"expected shape [n, {shape_tail}], got {tuple(t.shape)}")
    return t.data_ptr()


def _host_f32(a) -> np.ndarray:
    a = np.ascontiguousarray(a, dtype=np.float32)
    if a.ndim != 2 or a.shape[1] != 3:
        raise ValueError("expected a [n, 3] array")
    return a


# ---- the C entry points, same names ---------------------------------------

def scgr_default_params(**overrides) -> scgr_params:
    p = scgr_params()
    _check(load().scgr_default_params(ctypes.byref(p)))
    for k, v in overrides.items():
        if not hasattr(p, k):
            raise AttributeError(k)
        setattr(p, k, v)
    return p


def scgr_create(params: scgr_params | None = None, stream=None) -> c_void_p:
    """stream: a torch.cuda.Stream, a raw cudaStream_t int, or None for the
    current torch stream."""
    L = load()
    if params is None:
        params = scgr_default_params()
    if stream is None:
        import torch
        stream = torch.cuda.current_stream().cuda_stream
    elif hasattr(stream, "cuda_stream"):
        stream = stream.cuda_stream
    out = c_void_p()
    st = L.scgr_create(ctypes.byref(params), c_void_p(stream), ctypes.byref(out))
    _check(st, None)
    return out


def scgr_destroy(ctx) -> None:
    load().scgr_destroy(ctx)


def scgr_last_error(ctx) -> str:
    m = load().scgr_last_error(ctx)
    return m.decode() if m else ""


def scgr_set_reference(ctx, xyz) -> None:
    _check(load().scgr_set_reference(ctx, _dev_ptr(xyz, "float32", (3,)), xyz.shape[0]), ctx)


def scgr_set_template(ctx, xyz) -> None:
    _check(load().scgr_set_template(ctx, _dev_ptr(xyz, "float32", (3,)), xyz.shape[0]), ctx)


def scgr_set_reference_host(ctx, xyz) -> None:
    a = _host_f32(xyz)
    _check(load().scgr_set_reference_host(ctx, a.ctypes.data, a.shape[0]), ctx)


def scgr_set_template_host(ctx, xyz) -> None:
    a = _host_f32(xyz)
    _check(load().scgr_set_template_host(ctx, a.ctypes.data, a.shape[0]), ctx)


def scgr_compute_descriptors(ctx) -> None:
    _check(load().scgr_compute_descriptors(ctx), ctx)


def scgr_run(ctx, iterations: int) -> None:
    _check(load().scgr_run(ctx, int(iterations)), ctx)


def scgr_get_result(ctx) -> scgr_result:
    r = scgr_result()
    _check(load().scgr_get_result(ctx, ctypes.byref(r)), ctx)
    return r


def scgr_get_moved(ctx, out) -> None:
    _check(load().scgr_get_moved(ctx, _dev_ptr(out, "float32", (3,))), ctx)


def scgr_get_moved_host(ctx, out: np.ndarray) -> None:
    if out.dtype != np.float32 or not out.flags.c_contiguous or out.ndim != 2 or out.shape[1] != 3:
        raise ValueError("out must be a contiguous float32 [m, 3] array")
    _check(load().scgr_get_moved_host(ctx, out.ctypes.data), ctx)


def scgr_get_descriptors(ctx, which: int, knn_out=None, a_out=None) -> None:
    kp = _dev_ptr(knn_out, "int32") if knn_out is not None else None
    ap = _dev_ptr(a_out, "float32") if a_out is not None else None
    _check(load().scgr_get_descriptors(ctx, which, kp, ap), ctx)


def scgr_get_curvature64(ctx, which: int, out) -> None:
    _check(load().scgr_get_curvature64(ctx, which, _dev_ptr(out, "float64")), ctx)


def scgr_get_sigma(ctx) -> float:
    v = c_double()
    _check(load().scgr_get_sigma(ctx, ctypes.byref(v)), ctx)
    return v.value


def scgr_set_curvature(ctx, which: int, a64) -> None:
    _check(load().scgr_set_curvature(ctx, which, _dev_ptr(a64, "float64")), ctx)


def scgr_set_force_timing(ctx, enable: bool) -> None:
    _check(load().scgr_set_force_timing(ctx, 1 if enable else 0), ctx)


def scgr_get_force_timing(ctx):
    n = c_int64()
    ms = c_double()
    _check(load().scgr_get_force_timing(ctx, ctypes.byref(n), ctypes.byref(ms)), ctx)
    return int(n.value), float(ms.value)


def scgr_forces_static(x, y, ax, ay, f4_out, sigma: float = 0.0, p: float = 1.0, g_mode: int = 1,
                       stream=None) -> None:
    """Allocation-free force evaluation (no context): for callers that cannot
    allocate device memory.  x [n,3] / y [m,3] float32, ax [n] / ay [m]
    float64, f4_out [m,4] float32, all CUDA tensors; at most 131072 points
    per cloud; synchronises the stream."""
    if stream is None:
        import torch
        stream = torch.cuda.current_stream().cuda_stream
    elif hasattr(stream, "cuda_stream"):
        stream = stream.cuda_stream
    st = load().scgr_forces_static(_dev_ptr(x, "float32", (3,)), x.shape[0], _dev_ptr(y, "float32", (3,)),
                                   y.shape[0], _dev_ptr(ax, "float64"), _dev_ptr(ay, "float64"), float(sigma),
                                   float(p), int(g_mode), _dev_ptr(f4_out, "float32", (4,)), c_void_p(stream))
    if st != SCGR_OK:
        raise ScgrError(st, "scgr_forces_static failed")


def scgr_potential(ctx, pose7, want_grad: bool = True, grad_xyz_out=None):
    """U at pose7 = (omega, t, s); with want_grad also dU/dpose7 (numpy
    float64[7]); grad_xyz_out (CUDA float32 [m,3]) receives dU/dY0."""
    p7 = (c_double * 7)(*[float(v) for v in np.asarray(pose7, dtype=np.float64).reshape(7)])
    U = c_double()
    g7 = (c_double * 7)() if want_grad else None
    gx = _dev_ptr(grad_xyz_out, "float32", (3,)) if grad_xyz_out is not None else None
    _check(load().scgr_potential(ctx, p7, ctypes.byref(U), g7, gx), ctx)
    return float(U.value), (np.array(g7[:]) if want_grad else None)


def scgr_batch_run(ctx, ref_off, ref_xyz, tmp_off, tmp_xyz, iterations: int):
    """npairs registrations in one call.  ref_off/tmp_off: host int64 arrays of
    npairs + 1 offsets; ref_xyz/tmp_xyz: CUDA float32 [total, 3] tensors.
    Returns a list of scgr_result."""
    ro = np.ascontiguousarray(ref_off, dtype=np.int64)
    to = np.ascontiguousarray(tmp_off, dtype=np.int64)
    npairs = len(ro) - 1
    if len(to) != npairs + 1:
        raise ValueError("offset arrays differ in length")
    res = (scgr_result * npairs)()
    _check(load().scgr_batch_run(ctx, npairs, ro.ctypes.data, _dev_ptr(ref_xyz, "float32", (3,)), to.ctypes.data,
                                 _dev_ptr(tmp_xyz, "float32", (3,)), int(iterations), ctypes.addressof(res)), ctx)
    return list(res)


def scgr_set_row_range(ctx, row0: int, rows: int) -> None:
    _check(load().scgr_set_row_range(ctx, int(row0), int(rows)), ctx)


def scgr_step_partials(ctx) -> np.ndarray:
    out = (c_double * 13)()
    _check(load().scgr_step_partials(ctx, out), ctx)
    return np.array(out[:])


def scgr_step_apply(ctx, totals) -> None:
    t = (c_double * 13)(*[float(v) for v in np.asarray(totals, dtype=np.float64).reshape(13)])
    _check(load().scgr_step_apply(ctx, t), ctx)


def scgr_step_partials_dev(ctx, out13) -> None:
    """Enqueue this rank's 13 float64 partial sums into the CUDA tensor out13
    (13 doubles, contiguous)."""
    if out13.numel() != 13:
        raise ValueError("out13 must hold 13 doubles")
    _check(load().scgr_step_partials_dev(ctx, _dev_ptr(out13.reshape(-1), "float64")), ctx)


def scgr_step_apply_dev(ctx, parts) -> None:
    """Enqueue the pose update from the ranks' partial sums gathered in rank
    order: a CUDA float64 tensor of shape [nparts, 13] (or 13 * nparts)."""
    if parts.numel() % 13 != 0 or parts.numel() == 0:
        raise ValueError("parts must hold nparts x 13 doubles")
    _check(load().scgr_step_apply_dev(ctx, _dev_ptr(parts.reshape(-1), "float64"), parts.numel() // 13), ctx)


def scgr_microbench(kind: int, stream=None):
    """(lane_ops, ms) of one throughput-microbenchmark launch filling the GPU:
    kind 0 FFMA, 1 fma.f32x2, 2 ex2, 3 sqrt, 4 lg2, 5 rsqrt, 6 ex2 and rsqrt
    interleaved, 7 the force kernel's mix (6 fma.f32x2 + ex2 + sqrt per step;
    counts steps)."""
    import torch
    blocks = 8 * torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    out = torch.empty(blocks * 256, dtype=torch.float32, device="cuda")
    if stream is None:
        stream = torch.cuda.current_stream().cuda_stream
    ops = c_int64()
    ms = c_double()
    st = load().scgr_microbench(int(kind), blocks, _dev_ptr(out, "float32"), c_void_p(stream), ctypes.byref(ops),
                                ctypes.byref(ms))
    if st != SCGR_OK:
        raise ScgrError(st, "scgr_microbench failed")
    return int(ops.value), float(ms.value)


def scgr_get_plan(ctx) -> dict:
    out = (c_int * 5)()
    _check(load().scgr_get_plan(ctx, out), ctx)
    return {"P": out[0], "tpb": out[1], "splits": out[2], "iblocks": out[3], "occ": out[4]}


def scgr_plan_preview(n: int, m: int, p: float, num_sms: int, blocks_per_sm: int) -> dict:
    out = (c_int * 7)()
    _check(load().scgr_plan_preview(c_int64(int(n)), c_int64(int(m)), c_double(float(p)), int(num_sms),
                                    int(blocks_per_sm), out))
    return {"P": out[0], "tpb": out[1], "occ": out[2], "splits": out[3], "tiles_per_split": out[4],
            "iblocks": out[5], "half": out[6]}


def scgr_set_tuning(ctx, key: int, value: int) -> None:
    _check(load().scgr_set_tuning(ctx, int(key), int(value)), ctx)


def scgr_debug_fail_allocations(count: int) -> None:
    _check(load().scgr_debug_fail_allocations(int(count)))


def scgr_force_vjp(ctx, v, grad_out) -> None:
    _check(load().scgr_force_vjp(ctx, _dev_ptr(v, "float32", (3,)), _dev_ptr(grad_out, "float32", (3,))), ctx)


def scgr_nearest(ctx, q, idx_out=None, key_out=None) -> None:
    _check(load().scgr_nearest(ctx, _dev_ptr(q, "float32", (3,)), q.shape[0],
                               _dev_ptr(idx_out, "int32") if idx_out is not None else None,
                               _dev_ptr(key_out, "float32") if key_out is not None else None), ctx)


def scgr_change_mask(ctx, threshold: float, mask_out, dist_out=None) -> None:
    _check(load().scgr_change_mask(ctx, float(threshold), _dev_ptr(mask_out, "uint8"),
                                   _dev_ptr(dist_out, "float32") if dist_out is not None else None), ctx)


def scgr_set_neighbourhood(ctx, k: int = 16, radius_scale: float = 1.0, sigma_scale: float = 1.0) -> None:
    _check(load().scgr_set_neighbourhood(ctx, int(k), float(radius_scale), float(sigma_scale)), ctx)


def run_pyramid(ctx, levels):
    """Pyramidal schedule: `levels` is a sequence of (iterations, k,
    radius_scale, sigma_scale); descriptors are recomputed at the start of
    each level and the registration continues from the current pose."""
    for iters, k, rscale, sscale in levels:
        scgr_set_neighbourhood(ctx, k, rscale, sscale)
        scgr_run(ctx, iters)
    return scgr_get_result(ctx)


def scgr_potential_stored(ctx, pose7, want_grad: bool = True, grad_xyz_out=None):
    """As scgr_potential, with the forward pass storing the N x M pair
    weights and the backward pass reading them (comparison variant)."""
    p7 = (c_double * 7)(*[float(v) for v in np.asarray(pose7, dtype=np.float64).reshape(7)])
    U = c_double()
    g7 = (c_double * 7)() if want_grad else None
    gx = _dev_ptr(grad_xyz_out, "float32", (3,)) if grad_xyz_out is not None else None
    _check(load().scgr_potential_stored(ctx, p7, ctypes.byref(U), g7, gx), ctx)
    return float(U.value), (np.array(g7[:]) if want_grad else None)


def scgr_forces(ctx, f4_out) -> None:
    _check(load().scgr_forces(ctx, _dev_ptr(f4_out, "float32", (4,))), ctx)


def scgr_get_state(ctx) -> scgr_state:
    s = scgr_state()
    _check(load().scgr_get_state(ctx, ctypes.byref(s)), ctx)
    return s


def scgr_set_state(ctx, state: scgr_state) -> None:
    _check(load().scgr_set_state(ctx, ctypes.byref(state)), ctx)


def scgr_sync(ctx) -> None:
    _check(load().scgr_sync(ctx), ctx)


def scgr_launch_count(ctx) -> int:
    return int(load().scgr_launch_count(ctx))


# ---- autograd ----------------------------------------------------------------

def _potential_function():
    import torch

    class Potential(torch.autograd.Function):
        """U(pose7, Y0) on a context whose template is Y0 (descriptors fixed).

        forward: the potential only; backward: the hand-written adjoint
        (scgr_potential with gradients), which recomputes the pair tiles
        instead of storing the N x M pair terms."""

        @staticmethod
        def forward(fctx, pose7, Y0, handle):
            fctx.handle = handle
            fctx.save_for_backward(pose7)
            fctx.m = Y0.shape[0]
            fctx.device = Y0.device
            U, _ = scgr_potential(handle, pose7.detach().double().cpu().numpy(), want_grad=False)
            return torch.tensor(U, dtype=torch.float64)

        @staticmethod
        def backward(fctx, gU):
            (pose7,) = fctx.saved_tensors
            gx = torch.empty((fctx.m, 3), dtype=torch.float32, device=fctx.device)
            _, g7 = scgr_potential(fctx.handle, pose7.detach().double().cpu().numpy(), want_grad=True,
                                   grad_xyz_out=gx)
            g = float(gU)
            gp = torch.from_numpy(g7).to(pose7.dtype) * g
            return gp.to(pose7.device), (gx * g).to(fctx.device), None

    return Potential


_POTENTIAL = None


def potential(pose7, Y0, handle):
    """Differentiable U(pose7, Y0): torch.autograd.Function around the
    hand-written adjoint.  `handle` is a context whose template is Y0."""
    global _POTENTIAL
    if _POTENTIAL is None:
        _POTENTIAL = _potential_function()
    return _POTENTIAL.apply(pose7, Y0, handle)


# ---- convenience wrapper ----------------------------------------------------

class Registration:
    """Owns one context.  `register(X, Y0, iterations)` runs the whole method
    on device tensors and returns (R, t, s) as numpy float64."""

    def __init__(self, params: scgr_params | None = None, stream=None, **overrides):
        if params is None:
            params = scgr_default_params(**overrides)
        self.params = params
        self.ctx = scgr_create(params, stream)

    def close(self):
        if self.ctx is not None:
            scgr_destroy(self.ctx)
            self.ctx = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_clouds(self, X, Y0):
        self.m = int(Y0.shape[0])
        scgr_set_reference(self.ctx, X)
        scgr_set_template(self.ctx, Y0)
        scgr_compute_descriptors(self.ctx)

    def register(self, X, Y0, iterations: int):
        self.set_clouds(X, Y0)
        scgr_run(self.ctx, iterations)
        return scgr_get_result(self.ctx).as_numpy()

    def forces(self):
        import torch
        f4 = torch.empty((self.m, 4), dtype=torch.float32, device="cuda")
        scgr_forces(self.ctx, f4)
        return f4
