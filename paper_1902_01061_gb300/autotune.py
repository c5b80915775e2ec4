"""Autotuner of the force kernel's tile shape and the batched work-item size.

Candidates are timed on the caller's inputs through the C ABI, with CUDA
events around each force launch on the library's own stream
(scgr_set_force_timing).  The winner is cached in a JSON file keyed by GPU
name, a power-of-two size bucket and the distance-exponent mode, so that a
later registration of a similar size picks it up with `apply_cached`.
Cache file: $SCGR_TUNE_CACHE, else ~/.cache/scgr/tune.json.
"""
from __future__ import annotations

import json
import math
import os
import time

from . import scgr

SINGLE_CANDIDATES = [(P, tpb, occ) for P in (1, 2, 4) for tpb in (128, 256) for occ in (0, 1)
                     if not (P == 4 and tpb == 256 and occ == 1)] + [(4, 128, 2), (2, 256, 2)]
BATCH_CHUNKS = (8, 16, 32)
BATCH_P = (0, 1, 2, 4)


def cache_path() -> str:
    return os.environ.get("SCGR_TUNE_CACHE", os.path.join(os.path.expanduser("~"), ".cache", "scgr", "tune.json"))


def _load() -> dict:
    try:
        with open(cache_path()) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _store(key: str, value: dict) -> None:
    data = _load()
    data[key] = value
    path = cache_path()
    os.makedirs(os.path.dirname(path), exist_ok=True)
    tmp = path + f".{os.getpid()}.tmp"
    with open(tmp, "w") as f:
        json.dump(data, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def _bucket(v: int) -> int:
    return int(round(math.log2(max(int(v), 1))))


def _pmode(p: float) -> str:
    return {1.0: "p1", 2.0: "p2", 3.0: "p3"}.get(float(p), "pgen")


def single_key(gpu: str, n: int, m: int, p: float) -> str:
    return f"{gpu}|single|n2^{_bucket(n)}|m2^{_bucket(m)}|{_pmode(p)}"


def batch_key(gpu: str, npairs: int, work: int, p: float) -> str:
    return f"{gpu}|batch|pairs2^{_bucket(npairs)}|work2^{_bucket(work)}|{_pmode(p)}"


def gpu_name() -> str:
    import torch
    return torch.cuda.get_device_name()


def time_forces(ctx, m: int, reps: int = 3) -> float:
    """Mean device time (ms) of the force kernel over `reps` force
    evaluations of a context with m template rows."""
    import torch
    f4 = torch.empty((m, 4), dtype=torch.float32, device="cuda")
    scgr.scgr_forces(ctx, f4)                      # warm
    scgr.scgr_set_force_timing(ctx, True)
    try:
        for _ in range(reps):
            scgr.scgr_forces(ctx, f4)
        n, ms = scgr.scgr_get_force_timing(ctx)
    finally:
        scgr.scgr_set_force_timing(ctx, False)
    return ms / max(n, 1)


def _apply(ctx, P: int, tpb: int, occ: int, rsq: int = 0, exo: int = 0) -> None:
    scgr.scgr_set_tuning(ctx, scgr.SCGR_TUNE_FORCE_P, P)
    scgr.scgr_set_tuning(ctx, scgr.SCGR_TUNE_FORCE_TPB, tpb)
    scgr.scgr_set_tuning(ctx, scgr.SCGR_TUNE_FORCE_OCC, occ)
    scgr.scgr_set_tuning(ctx, scgr.SCGR_TUNE_FORCE_RSQRT, rsq)
    scgr.scgr_set_tuning(ctx, scgr.SCGR_TUNE_FORCE_EX2POLY, exo)


def tune_single(ctx, n: int, m: int, p: float, candidates=None, reps: int = 3, store: bool = True) -> dict:
    """Time each (P, threads, occupancy variant) candidate on a context whose
    descriptors are computed (splits stay automatic); for p = 2 the two best
    shapes are timed again with the rsqrt form of the distance factor, and
    the best shared-memory-sum shape with part of its exponentials on the
    FP32 pipe (SCGR_TUNE_FORCE_EX2POLY 1 and 2).  Leave the best in place and
    return it."""
    results = []
    for P, tpb, occ in candidates or SINGLE_CANDIDATES:
        _apply(ctx, P, tpb, occ, 0)
        results.append((time_forces(ctx, m, reps), P, tpb, occ, 0, 0, scgr.scgr_get_plan(ctx)))
    results.sort(key=lambda r: r[0])
    if float(p) == 2.0:
        for r in results[:2]:
            _apply(ctx, r[1], r[2], r[3], 1)
            results.append((time_forces(ctx, m, reps), r[1], r[2], r[3], 1, 0, scgr.scgr_get_plan(ctx)))
        ks = [r for r in results if r[3] == 2 and r[4] == 0 and r[5] == 0]
        if ks:
            r = min(ks, key=lambda x: x[0])
            for exo in (1, 2):
                _apply(ctx, r[1], r[2], r[3], 0, exo)
                results.append((time_forces(ctx, m, reps), r[1], r[2], r[3], 0, exo, scgr.scgr_get_plan(ctx)))
        results.sort(key=lambda r: r[0])
    best_ms, P, tpb, occ, rsq, exo, plan = results[0]
    _apply(ctx, P, tpb, occ, rsq, exo)
    best = {"P": P, "tpb": tpb, "occ": occ, "rsqrt": rsq, "ex2poly": exo, "ms": best_ms, "plan": plan,
            "tried": [{"P": r[1], "tpb": r[2], "occ": r[3], "rsqrt": r[4], "ex2poly": r[5], "ms": r[0]}
                      for r in results],
            "when": time.strftime("%Y-%m-%d %H:%M:%S")}
    if store:
        _store(single_key(gpu_name(), n, m, p), best)
    return best


def tune_batch(ctx, ref_off, ref_xyz, tmp_off, tmp_xyz, p: float, iterations: int = 3, store: bool = True) -> dict:
    """Time scgr_batch_run for each work-item chunk length and points per
    thread, then the best of those with the persistent force kernel (and, for
    p = 2, with the rsqrt distance form); leave the best."""
    import numpy as np
    import torch
    ro = np.asarray(ref_off, dtype=np.int64)
    to = np.asarray(tmp_off, dtype=np.int64)
    work = int(np.sum(np.diff(ro) * np.diff(to)))

    def timed(ct, P, rsq, pers):
        scgr.scgr_set_tuning(ctx, scgr.SCGR_TUNE_BATCH_P, P)
        scgr.scgr_set_tuning(ctx, scgr.SCGR_TUNE_BATCH_CHUNK_TILES, ct)
        scgr.scgr_set_tuning(ctx, scgr.SCGR_TUNE_FORCE_RSQRT, rsq)
        scgr.scgr_set_tuning(ctx, scgr.SCGR_TUNE_BATCH_PERSISTENT, pers)
        scgr.scgr_batch_run(ctx, ro, ref_xyz, to, tmp_xyz, 1)           # warm
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        scgr.scgr_batch_run(ctx, ro, ref_xyz, to, tmp_xyz, iterations)
        return (time.perf_counter() - t0, ct, P, rsq, pers)

    results = [timed(ct, P, 0, 0) for P in BATCH_P for ct in BATCH_CHUNKS]
    results.sort()
    _, ct, P, _, _ = results[0]
    if P != 0:                                     # the mixed form has no persistent variant
        results.append(timed(ct, P, 0, 1))
    if float(p) == 2.0:
        results.append(timed(ct, P, 1, 0))
    results.sort()
    best_s, ct, P, rsq, pers = results[0]
    scgr.scgr_set_tuning(ctx, scgr.SCGR_TUNE_BATCH_P, P)
    scgr.scgr_set_tuning(ctx, scgr.SCGR_TUNE_BATCH_CHUNK_TILES, ct)
    scgr.scgr_set_tuning(ctx, scgr.SCGR_TUNE_FORCE_RSQRT, rsq)
    scgr.scgr_set_tuning(ctx, scgr.SCGR_TUNE_BATCH_PERSISTENT, pers)
    best = {"chunk_tiles": ct, "P": P, "rsqrt": rsq, "persistent": pers, "s": best_s, "iterations": iterations,
            "tried": [{"chunk_tiles": c, "P": q, "rsqrt": r, "persistent": e, "s": t} for t, c, q, r, e in results],
            "when": time.strftime("%Y-%m-%d %H:%M:%S")}
    if store:
        _store(batch_key(gpu_name(), len(ro) - 1, work, p), best)
    return best


def apply_cached_single(ctx, n: int, m: int, p: float) -> dict | None:
    hit = _load().get(single_key(gpu_name(), n, m, p))
    if hit:
        _apply(ctx, hit["P"], hit["tpb"], hit.get("occ", 0), hit.get("rsqrt", 0), hit.get("ex2poly", 0))
    return hit


def apply_cached_batch(ctx, npairs: int, work: int, p: float) -> dict | None:
    hit = _load().get(batch_key(gpu_name(), npairs, work, p))
    if hit:
        scgr.scgr_set_tuning(ctx, scgr.SCGR_TUNE_BATCH_CHUNK_TILES, hit["chunk_tiles"])
        scgr.scgr_set_tuning(ctx, scgr.SCGR_TUNE_BATCH_P, hit.get("P", 1))
        scgr.scgr_set_tuning(ctx, scgr.SCGR_TUNE_FORCE_RSQRT, hit.get("rsqrt", 0))
        scgr.scgr_set_tuning(ctx, scgr.SCGR_TUNE_BATCH_PERSISTENT, hit.get("persistent", 0))
    return hit
