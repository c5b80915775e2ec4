#!/usr/bin/env python3
"""Benchmark of the registration hot path on GB300.

One step = one whole registration of the benchmark workload through the C
ABI: pack + validate both clouds, the kNN/curvature descriptor pass, the
iterations (all-pairs force, combine, float64 pose update) and the moved
template.  Default workload: 1,000,000 template x 1,000,000 reference points
(8-ellipsoid surface with a 15% box-shaped outlier cluster), p = 2,
g = aX aY s, k = 16, 50 iterations: 5e13 pair interactions per step.

Prints one JSON line.  `value` is pair-interactions/s over the device-timed
steps (inputs resident in HBM); `e2e` repeats the steps through the host
entry points with pinned host buffers (host->device copies and the moved
cloud's device->host copy inside the timed region).  `roofline` reports the
force kernel against the FP32 issue peak (2 x 128 lanes x SMs x max clock);
`cpu_baseline` times the FP64 oracle on a bounded sample on the host cores.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

# counting convention of the per-pair work: r = Y - X (3), d^2 (5), d^(p-1) (1),
# the similarity exponent and exp (4), x aX (1), x d^(p-1) (1), W (1), f (6)
FLOPS_PER_PAIR = 22
FP32_LANES_PER_SM = 128
L2_FLUSH_BYTES = 256 << 20   # > 129 MB L2

WORKLOADS = {
    "large": dict(desc="1,000,000 template x 1,000,000 reference points, 8-ellipsoid surface, 15% box outlier "
                       "cluster, rotation 60 deg, scale 1.1, p=2, g=aX*aY*s, k=16, 50 iterations",
                  n=1_000_000, iters=50),
    "scale": dict(desc="35,000 reference x 30,800 template points (5-ellipsoid surface, 20% slab removed, "
                       "10% uniform outliers), p=2, k=16, 200 iterations", n=35_000, iters=200),
    "mid": dict(desc="320,000 template x 320,000 reference points from the large-case generator, p=2, k=16, "
                     "5 iterations (small case for profiler captures)", n=320_000, iters=5),
    "tiny": dict(desc="1,000 x 1,000 points (3-ellipsoid surface, 50 deg about x), p=2, k=16, 100 iterations",
                 n=1000, iters=100),
}


def metric_name(workload):
    return "pair-interactions/s at 1Mx1M" if workload == "large" else "pair-interactions/s"


def base_config(workload, n, m):
    wl = WORKLOADS[workload]
    return {"workload": wl["desc"], "N": n, "M": m, "iterations": wl["iters"], "p": 2.0, "g_mode": 1, "k": 16,
            "pairs_per_step": n * m * wl["iters"]}


def make_pair(name):
    from paper_1902_01061_gb300 import synth
    if name == "large":
        return synth.large_case()
    if name == "scale":
        return synth.scale_case()
    if name == "mid":
        return synth.large_case(n=320_000)
    return synth.tiny()


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int | None):
        self.proc = None
        self.lines = []
        self.gpu_index = gpu_index

    def start(self):
        cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "200"]
        if self.gpu_index is not None:
            cmd += ["-i", str(self.gpu_index)]
        try:
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "samples": len(sm),
                "reasons": sorted(reasons)}


def gpu_index_for(local_rank: int):
    vis = os.environ.get("CUDA_VISIBLE_DEVICES")
    if vis:
        items = [v.strip() for v in vis.split(",") if v.strip()]
        if local_rank < len(items) and items[local_rank].isdigit():
            return int(items[local_rank])
        return None
    return local_rank


def profile_traffic():
    """Per-launch DRAM bytes of the force kernel from the committed ncu summary,
    or None when the kernel source changed since the counters were taken."""
    path = os.path.join(ROOT, "profiles", "force_tile_kernel_large.md")
    src = os.path.join(ROOT, "paper_1902_01061_gb300", "csrc", "force.cu")
    if not (os.path.exists(path) and os.path.exists(src)):
        return None, None
    digest = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
    traffic, tag = None, None
    for line in open(path):
        if line.startswith("traffic_bytes_per_launch_full_size:"):
            traffic = float(line.split(":", 1)[1].split()[0])
        if line.startswith("force_cu_sha256_16:"):
            tag = line.split(":", 1)[1].strip()
    return (traffic if tag == digest else None), digest


def measured_peaks(scgr, num_sms, sm_mhz):
    """Unit throughputs measured by the library's microbenchmark at the
    current clock: FP32 lane-FMAs and MUFU results per clock per SM."""
    names = ["ffma", "ffma2_f32x2", "mufu_ex2", "mufu_sqrt", "mufu_lg2", "mufu_rsqrt", "mufu_ex2_rsqrt_mixed",
             "mix_6ffma2_ex2_sqrt"]
    out = {}
    for kind, name in enumerate(names):
        ops, ms = scgr.scgr_microbench(kind)
        per_clk_sm = ops / (ms * 1e-3) / (num_sms * sm_mhz * 1e6)
        out[name] = {"per_clk_per_sm": per_clk_sm, "ms": ms}
        if kind <= 1:
            out[name]["tflops"] = 2 * ops / (ms * 1e-3) / 1e12
    out["clock_mhz_assumed"] = sm_mhz
    return out


def cpu_baseline(pair, p, g_mode, seconds=15.0):
    """The FP64 oracle as it stands, on the host, for a bounded sample: the
    iteration-0 force pass (Eq. 5) for a few template rows against every
    reference point.  Curvatures are seeded synthetic values (timing only)."""
    import numpy as np
    import oracle as O
    rng = np.random.default_rng(1234)
    n, m = len(pair.X), len(pair.Y0)
    aX = np.clip(rng.gamma(1.2, 0.015, size=n), 0, 0.33)
    aY = np.clip(rng.gamma(1.2, 0.015, size=m), 0, 0.33)
    sigma = O.sigma_auto(aX)
    Y = pair.Y0.astype(np.float64)
    probe = np.arange(4)
    t0 = time.perf_counter()
    O.forces_rows(Y, pair.X, aY, aX, sigma, p, g_mode, probe)
    per_row = (time.perf_counter() - t0) / len(probe)
    nrows = int(max(4, min(m, seconds / max(per_row, 1e-9))))
    rows = np.sort(rng.choice(m, size=nrows, replace=False))
    t0 = time.perf_counter()
    O.forces_rows(Y, pair.X, aY, aX, sigma, p, g_mode, rows)
    dt = time.perf_counter() - t0
    value = nrows * n / dt
    out = {"value": value, "unit": "pair-interactions/s", "cores": 1, "kind": "oracle",
           "sample": f"iteration-0 force pass (Eq. 5) of {nrows} template rows x {n} reference points "
                     f"in float64 numpy, single thread, {dt:.1f} s",
           "cpu": _cpu_model(), "nproc": os.cpu_count() or 1,
           "extrapolated_s_per_iteration": n * m / value}
    try:
        allc = cpu_baseline_all_cores(pair, p, g_mode, dt / nrows)
        allc["extrapolated_s_per_iteration"] = n * m / allc["value"]
        out["all_cores"] = allc
    except Exception as e:                       # the single-thread figure stands on its own
        out["all_cores"] = {"unavailable": f"{type(e).__name__}: {e}"[:200]}
    return out


# Arm CPU part numbers (implementer 0x41) of the Neoverse cores that hosts
# of this class carry; /proc/cpuinfo on Arm gives only the part number.
ARM_PARTS = {"0xd0c": "Neoverse-N1", "0xd40": "Neoverse-V1", "0xd49": "Neoverse-N2", "0xd4f": "Neoverse-V2",
             "0xd84": "Neoverse-V3", "0xd8e": "Neoverse-N3"}


def _cpu_model():
    """Host CPU model name, e.g. 'Neoverse-V2 (Arm part 0xd4f)' on an Arm host
    or the 'model name' line on x86."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().lower().startswith("model name"):
                name = line.split(":", 1)[1].strip()
                if name and name != "-":
                    return name
    except (OSError, subprocess.SubprocessError):
        pass
    fields = {}
    try:
        for line in open("/proc/cpuinfo"):
            if ":" in line:
                k, v = line.split(":", 1)
                fields.setdefault(k.strip().lower(), v.strip())
    except OSError:
        pass
    if "model name" in fields:
        return fields["model name"]
    part = fields.get("cpu part")
    if part:
        name = ARM_PARTS.get(part.lower()) if fields.get("cpu implementer", "").lower() == "0x41" else None
        return f"{name} (Arm part {part})" if name else f"Arm part {part}"
    import platform
    return platform.processor() or platform.machine()


def _host_info():
    return {"cpu": _cpu_model(), "nproc": os.cpu_count() or 1}


_POOL_DATA = {}


def _pool_init(Y, X, aY, aX, sigma, p, g_mode):
    os.environ.setdefault("OMP_NUM_THREADS", "1")
    _POOL_DATA.update(Y=Y, X=X, aY=aY, aX=aX, sigma=sigma, p=p, g_mode=g_mode)


def _pool_rows(rows):
    import oracle as O
    d = _POOL_DATA
    O.forces_rows(d["Y"], d["X"], d["aY"], d["aX"], d["sigma"], d["p"], d["g_mode"], rows)
    return len(rows)


def cpu_baseline_all_cores(pair, p, g_mode, per_row_s, seconds=10.0):
    """The same oracle sample spread over every host core: a spawned process
    pool (started fresh, so no CUDA state is inherited), one block of template
    rows per process, each row summed as the oracle sums it."""
    import multiprocessing as mp
    import numpy as np
    import oracle as O
    cores = os.cpu_count() or 1
    rng = np.random.default_rng(4321)
    n, m = len(pair.X), len(pair.Y0)
    aX = np.clip(rng.gamma(1.2, 0.015, size=n), 0, 0.33)
    aY = np.clip(rng.gamma(1.2, 0.015, size=m), 0, 0.33)
    sigma = O.sigma_auto(aX)
    Y = pair.Y0.astype(np.float64)
    per_core = int(max(2, seconds / max(per_row_s, 1e-9)))
    rows = np.sort(rng.choice(m, size=min(m, per_core * cores), replace=False))
    chunks = np.array_split(rows, cores)
    ctx = mp.get_context("spawn")
    with ctx.Pool(cores, initializer=_pool_init, initargs=(Y, pair.X, aY, aX, sigma, p, g_mode)) as pool:
        pool.map(_pool_rows, [c[:1] for c in chunks])          # workers up, oracle imported
        t0 = time.perf_counter()
        done = sum(pool.map(_pool_rows, chunks))
        dt = time.perf_counter() - t0
    return {"value": done * n / dt, "unit": "pair-interactions/s", "cores": cores, "kind": "oracle",
            "sample": f"iteration-0 force pass of {done} template rows x {n} reference points, float64 numpy, "
                      f"{cores} spawned processes over row blocks, {dt:.1f} s"}


def oracle_runs():
    """The FP64 oracle, as it stands, on the two configurations a host can
    run end to end.  Config 1 (1,000 x 1,000, p = 2, 100 iterations): the
    full registration (descriptors + iterations) on one thread, and with each
    iteration's force rows spread over a spawned process pool of every core
    (row blocks added in block order, `register_from_partials`).  Config 2
    (35,000 x 30,800, p = 2, 200 iterations): the descriptor pass timed in
    full, one whole iteration timed on every core, and one iteration's force
    pass on one thread timed on a 1-in-64 row sample; the 200-iteration
    totals are extrapolated from those (a full run takes hours on one
    thread)."""
    import multiprocessing as mp
    import numpy as np
    import oracle as O
    from paper_1902_01061_gb300 import synth
    cores = os.cpu_count() or 1
    prm = O.Params(p=2.0)
    out = {"kind": "oracle", "cpu": _cpu_model(), "nproc": cores}
    t = synth.tiny()
    t0 = time.perf_counter()
    d = O.descriptors(t.X, t.Y0, prm)
    O.register(t.X, t.Y0, prm, iterations=100, desc=d)
    one = time.perf_counter() - t0
    sc = synth.scale_case()
    with mp.get_context("spawn").Pool(cores) as pool:
        slim = {"aX": d["aX"], "aY": d["aY"], "sigma": d["sigma"]}
        blocks = np.array_split(np.arange(len(t.Y0)), cores)
        O.register_from_partials(t.X, t.Y0, prm, 1, slim, blocks, map_partials=pool.map)     # workers up
        t0 = time.perf_counter()
        d = O.descriptors(t.X, t.Y0, prm)
        O.register_from_partials(t.X, t.Y0, prm, 100, {"aX": d["aX"], "aY": d["aY"], "sigma": d["sigma"]}, blocks,
                                 map_partials=pool.map)
        allc = time.perf_counter() - t0
        out["tiny_1k"] = {
            "workload": "1,000 x 1,000 points, p=2, k=16, 100 iterations (descriptors + iterations)",
            "s_single_thread": one, "s_all_cores": allc, "cores": cores,
            "pair_interactions_per_s_single_thread": 1000 * 1000 * 100 / one}
        t0 = time.perf_counter()
        d2 = O.descriptors(sc.X, sc.Y0, prm)
        desc_s = time.perf_counter() - t0
        slim2 = {"aX": d2["aX"], "aY": d2["aY"], "sigma": d2["sigma"]}
        blocks2 = np.array_split(np.arange(len(sc.Y0)), cores)
        t0 = time.perf_counter()
        O.register_from_partials(sc.X, sc.Y0, prm, 1, slim2, blocks2, map_partials=pool.map)
        it_all = time.perf_counter() - t0
    rows = np.arange(0, len(sc.Y0), 64)
    t0 = time.perf_counter()
    O.forces_rows(sc.Y0, sc.X, d2["aY"], d2["aX"], d2["sigma"], 2.0, 1, rows)
    it_one = (time.perf_counter() - t0) * len(sc.Y0) / len(rows)
    n2, m2 = len(sc.X), len(sc.Y0)
    out["scale_35k"] = {
        "workload": f"{n2:,} x {m2:,} points, p=2, k=16, 200 iterations",
        "descriptors_s": desc_s, "s_per_iteration_all_cores": it_all, "s_per_iteration_single_thread": it_one,
        "extrapolated_s_all_cores": desc_s + 200 * it_all, "extrapolated_s_single_thread": desc_s + 200 * it_one,
        "pair_interactions_per_s_all_cores": n2 * m2 / it_all, "cores": cores,
        "sample": "descriptors in full; one full iteration on every core; one thread on a 1-in-64 row sample"}
    return out


def bench_batch(args, scgr, torch, dev, steps, warmup):
    """Batched registrations/s on 512 pairs (log-uniform 500-20,000 points,
    rotation <= 90 deg, scale 0.7-1.4, 0-15% outliers), 100 iterations in one
    CUDA graph, against one call per pair (same parameters, graph per pair)."""
    import numpy as np
    from paper_1902_01061_gb300 import synth
    pairs = synth.batch_case()
    iters = getattr(args, "batch_iters", 100)
    ro = np.cumsum([0] + [len(pp.X) for pp in pairs]).astype(np.int64)
    to = np.cumsum([0] + [len(pp.Y0) for pp in pairs]).astype(np.int64)
    Xc = torch.from_numpy(np.concatenate([pp.X for pp in pairs])).to(dev)
    Yc = torch.from_numpy(np.concatenate([pp.Y0 for pp in pairs])).to(dev)
    pair_work = int(sum(len(pp.X) * len(pp.Y0) for pp in pairs))
    params = scgr.scgr_default_params(p=2.0, g_mode=1, k=16, use_graph=0 if getattr(args, "batch_eager", False) else 1)
    stream = torch.cuda.current_stream()
    ctx = scgr.scgr_create(params, stream)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    tuned = None
    if getattr(args, "batch_plan", None):
        vals = [int(v) for v in args.batch_plan.split(",")]
        bP, bC = vals[0], vals[1]
        bQ = vals[2] if len(vals) > 2 else 0
        scgr.scgr_set_tuning(ctx, scgr.SCGR_TUNE_BATCH_P, bP)
        scgr.scgr_set_tuning(ctx, scgr.SCGR_TUNE_BATCH_CHUNK_TILES, bC)
        scgr.scgr_set_tuning(ctx, scgr.SCGR_TUNE_BATCH_PERSISTENT, bQ)
        tuned = {"P": bP, "chunk_tiles": bC, "persistent": bQ, "pinned": True}
    elif not args.no_autotune:
        from paper_1902_01061_gb300 import autotune
        tuned = autotune.tune_batch(ctx, ro, Xc, to, Yc, 2.0, iterations=3)

    def one_batch():
        scgr.scgr_batch_run(ctx, ro, Xc, to, Yc, iters)

    for _ in range(warmup):
        one_batch()
    times = []
    l0 = scgr.scgr_launch_count(ctx)
    for _ in range(steps):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        one_batch()                      # synchronises (results copied to the host)
        times.append(time.perf_counter() - t0)
    batch_launches = (scgr.scgr_launch_count(ctx) - l0) // max(steps, 1)
    batch_s = sum(times) / len(times)
    dtimes = []                          # descriptors alone: the same call with 0 iterations
    for _ in range(max(steps, 1)):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        scgr.scgr_batch_run(ctx, ro, Xc, to, Yc, 0)
        dtimes.append(time.perf_counter() - t0)
    desc_s = sum(dtimes) / len(dtimes)
    scgr.scgr_destroy(ctx)

    out = {"workload": "512 pairs, 500-20,000 points log-uniform, rotation <= 90 deg, scale 0.7-1.4, "
                       f"0-15% outliers, p=2, k=16, {iters} iterations "
                       + ("with eager launches" if getattr(args, "batch_eager", False) else "in one CUDA graph"),
           "npairs": len(pairs), "points": int(ro[-1] + to[-1]), "pair_interactions_per_iteration": pair_work,
           "registrations_per_s": len(pairs) / batch_s, "ms_per_batch": batch_s * 1e3,
           "descriptors_ms": desc_s * 1e3,
           "registrations_per_s_without_descriptors": len(pairs) / max(batch_s - desc_s, 1e-9),
           "pair_interactions_per_s": pair_work * iters / batch_s,
           "launches_per_batch": int(batch_launches),
           "autotuned": tuned,
           "timing": "host wall clock around each synchronising call, L2 flushed before each"}
    if getattr(args, "batch_only", False):
        return out

    # one call per pair, same method parameters, eager launches (capturing a
    # graph per pair costs more than it saves at 100 iterations)
    ctx1 = scgr.scgr_create(scgr.scgr_default_params(p=2.0, g_mode=1, k=16), stream)
    views = [(Xc[ro[i]:ro[i + 1]], Yc[to[i]:to[i + 1]]) for i in range(len(pairs))]

    def per_pair():
        for xv, yv in views:
            scgr.scgr_set_reference(ctx1, xv)
            scgr.scgr_set_template(ctx1, yv)
            scgr.scgr_compute_descriptors(ctx1)
            scgr.scgr_run(ctx1, iters)
            scgr.scgr_get_result(ctx1)

    per_pair()                           # warm (graph instantiation for each size)
    flush.zero_()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    per_pair()
    single_s = time.perf_counter() - t0
    scgr.scgr_destroy(ctx1)
    out.update({"one_call_per_pair_registrations_per_s": len(pairs) / single_s,
                "speedup_vs_one_call_per_pair": single_s / batch_s,
                "one_call_per_pair": "scgr_set_reference/template + compute_descriptors + run(100) + get_result "
                                     "per pair, eager launches"})
    return out


def _timed(fn, steps, warmup, torch):
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    out = []
    for _ in range(steps):
        t0 = time.perf_counter()
        fn()
        torch.cuda.synchronize()
        out.append(time.perf_counter() - t0)
    return sum(out) / len(out)


def bench_diff(args, scgr, torch, dev, steps, warmup):
    """Differentiation form at 50,000 x 50,000 (rotation 30 deg, noise 0.01 of
    the diagonal): the potential alone, potential + adjoint with tile
    recomputation, and potential + adjoint from stored pair terms."""
    from paper_1902_01061_gb300 import synth
    nd = getattr(args, "diff_n", 50_000)
    case = synth.diff_case(n=nd)
    n, m = len(case.X), len(case.Y0)
    ctx = scgr.scgr_create(scgr.scgr_default_params(p=2.0), torch.cuda.current_stream())
    try:
        scgr.scgr_set_reference(ctx, torch.from_numpy(case.X).to(dev))
        scgr.scgr_set_template(ctx, torch.from_numpy(case.Y0).to(dev))
        scgr.scgr_compute_descriptors(ctx)
        tuned = None
        if not args.no_autotune:
            from paper_1902_01061_gb300 import autotune
            tuned = autotune.tune_single(ctx, n, m, 2.0, reps=10)
            tuned = {k: tuned[k] for k in ("P", "tpb", "occ", "rsqrt", "ex2poly", "ms", "plan")}
        pose = [0.1, -0.2, 0.3, 0.05, 0.0, -0.05, 1.02]
        gx = torch.empty((m, 3), dtype=torch.float32, device=dev)
        fwd = _timed(lambda: scgr.scgr_potential(ctx, pose, want_grad=False), steps, warmup, torch)
        both = _timed(lambda: scgr.scgr_potential(ctx, pose, grad_xyz_out=gx), steps, warmup, torch)
        stored = _timed(lambda: scgr.scgr_potential_stored(ctx, pose, grad_xyz_out=gx), steps, warmup, torch)
    finally:
        scgr.scgr_destroy(ctx)
    return {"workload": f"{n:,} x {m:,} points, rotation 30 deg, noise 0.01 of the diagonal, p=2",
            "potential_ms": fwd * 1e3, "potential_and_adjoint_recompute_ms": both * 1e3,
            "potential_and_adjoint_stored_ms": stored * 1e3,
            "stored_pair_terms_bytes": m * ((n + 255) // 256 * 256) * 4,
            "adjoint_pair_interactions_per_s": 2 * n * m / both, "autotuned": tuned,
            "timing": "host wall clock around each synchronising call"}


def bench_scale(args, scgr, torch, dev, steps, warmup):
    """One registration of the 35,000-point case (200 iterations) per step."""
    from paper_1902_01061_gb300 import synth
    case = synth.scale_case()
    n, m = len(case.X), len(case.Y0)
    X = torch.from_numpy(case.X).to(dev)
    Y = torch.from_numpy(case.Y0).to(dev)
    ctx = scgr.scgr_create(scgr.scgr_default_params(p=2.0, use_graph=1), torch.cuda.current_stream())
    tuned = None
    try:
        if not args.no_autotune:
            from paper_1902_01061_gb300 import autotune
            scgr.scgr_set_reference(ctx, X)
            scgr.scgr_set_template(ctx, Y)
            scgr.scgr_compute_descriptors(ctx)
            tuned = autotune.tune_single(ctx, n, m, 2.0, reps=10)
            tuned = {k: tuned[k] for k in ("P", "tpb", "occ", "rsqrt", "ex2poly", "ms", "plan")}

        def one():
            scgr.scgr_set_reference(ctx, X)
            scgr.scgr_set_template(ctx, Y)
            scgr.scgr_compute_descriptors(ctx)
            scgr.scgr_run(ctx, 200)
            scgr.scgr_get_result(ctx)
        sec = _timed(one, steps, warmup, torch)
    finally:
        scgr.scgr_destroy(ctx)
    return {"workload": "35,000 reference x 30,800 template points, 200 iterations, p=2, CUDA graph",
            "ms_per_registration": sec * 1e3, "pair_interactions_per_s": n * m * 200 / sec, "autotuned": tuned}


def bench_next(args, scgr, torch, dev, steps, warmup, Xd, Yd):
    """The widened rows, each timed once set up: the odd-p fast path on the
    1M x 1M workload (p = 1: pose-free force sums computed once per call;
    p = 3: 14 pose-free moments), and on the 35,000-point case the radius
    neighbourhood of Sec. IV, the pyramidal schedule and the change mask of
    Sec. V after registration."""
    from paper_1902_01061_gb300 import synth
    out = {}
    n, m = int(Xd.shape[0]), int(Yd.shape[0])
    stream = torch.cuda.current_stream()
    for p in (1.0, 3.0):
        ctx = scgr.scgr_create(scgr.scgr_default_params(p=p, g_mode=1, k=16), stream)
        try:
            scgr.scgr_set_reference(ctx, Xd)
            scgr.scgr_set_template(ctx, Yd)
            scgr.scgr_compute_descriptors(ctx)
            fast = _timed(lambda: (scgr.scgr_run(ctx, 50), scgr.scgr_get_result(ctx)), steps, 1, torch)
            if p == 1.0:
                # change mask (Sec. V) at full size: grid search of the 1M reference
                diag = float((Xd.max(dim=0).values - Xd.min(dim=0).values).norm().item())
                mask = torch.empty(m, dtype=torch.uint8, device=dev)
                chg = _timed(lambda: scgr.scgr_change_mask(ctx, 0.01 * diag, mask), steps, 1, torch)
                flagged = int(mask.sum().item())
                scgr.scgr_set_tuning(ctx, scgr.SCGR_TUNE_NEAREST_LEVELS, 1)
                chg1 = _timed(lambda: scgr.scgr_change_mask(ctx, 0.01 * diag, mask), 1, 1, torch)
                scgr.scgr_set_tuning(ctx, scgr.SCGR_TUNE_NEAREST_LEVELS, 2)
                out["change_mask_full_size"] = {
                    "workload": f"{m:,} moved template points against {n:,} reference points (exact two-level grid "
                                "search), threshold 1% of the diagonal, after the p = 1 registration",
                    "ms": chg * 1e3, "ms_fine_shells_only": chg1 * 1e3, "points_flagged": flagged}
            scgr.scgr_set_tuning(ctx, scgr.SCGR_TUNE_REUSE_POSE_FREE, 0)
            per_it = _timed(lambda: (scgr.scgr_run(ctx, 2), scgr.scgr_get_result(ctx)), 1, 1, torch) / 2
        finally:
            scgr.scgr_destroy(ctx)
        out[f"odd_p_fast_path_p{int(p)}"] = {
            "workload": f"{n:,} x {m:,}, p = {p:g}, 50 iterations",
            "ms_per_registration": fast * 1e3, "all_pairs_ms_per_iteration": per_it * 1e3,
            "speedup_vs_all_pairs_every_iteration": 50 * per_it / fast,
            "equivalent_pair_interactions_per_s": n * m * 50 / fast}
    sc = synth.scale_case()
    X = torch.from_numpy(sc.X).to(dev)
    Y = torch.from_numpy(sc.Y0).to(dev)
    ctx = scgr.scgr_create(scgr.scgr_default_params(p=2.0, neigh_mode=1, radius_scale=1.0), stream)
    try:
        scgr.scgr_set_reference(ctx, X)
        scgr.scgr_set_template(ctx, Y)
        rad = _timed(lambda: scgr.scgr_compute_descriptors(ctx), steps, 1, torch)
    finally:
        scgr.scgr_destroy(ctx)
    out["radius_neighbourhood"] = {"workload": "35,000 + 30,800 points, radius sqrt(e) (scale 1.0), both clouds",
                                   "ms_descriptors": rad * 1e3}
    levels = [(70, 24, 1.0, 1.5), (70, 16, 1.0, 1.0), (60, 8, 1.0, 0.7)]
    ctx = scgr.scgr_create(scgr.scgr_default_params(p=2.0, use_graph=1, E=200), stream)
    try:
        def pyramid():
            scgr.scgr_set_reference(ctx, X)
            scgr.scgr_set_template(ctx, Y)
            scgr.scgr_compute_descriptors(ctx)
            scgr.run_pyramid(ctx, levels)
        pyr = _timed(pyramid, steps, 1, torch)
        mask = torch.empty(len(sc.Y0), dtype=torch.uint8, device=dev)
        diag = float(synth.bbox_diag(sc.X))
        chg = _timed(lambda: scgr.scgr_change_mask(ctx, 0.01 * diag, mask), steps, 1, torch)
        changed = int(mask.sum().item())
    finally:
        scgr.scgr_destroy(ctx)
    out["pyramidal_schedule"] = {"workload": "35,000 x 30,800, levels (iterations, k, sigma scale) = "
                                             "(70, 24, 1.5), (70, 16, 1.0), (60, 8, 0.7), CUDA graph per level",
                                 "ms_per_registration": pyr * 1e3}
    out["change_mask"] = {"workload": "30,800 moved template points against 35,000 reference points, "
                                      "threshold 1% of the diagonal",
                          "ms": chg * 1e3, "points_flagged": changed}
    out["timing"] = "host wall clock around synchronised calls"
    return out


def apply_plan(scgr, ctx, tuned):
    """Pin the force plan the main leg's autotuner picked."""
    if tuned and "P" in tuned:
        scgr.scgr_set_tuning(ctx, scgr.SCGR_TUNE_FORCE_P, int(tuned["P"]))
        scgr.scgr_set_tuning(ctx, scgr.SCGR_TUNE_FORCE_TPB, int(tuned["tpb"]))
        scgr.scgr_set_tuning(ctx, scgr.SCGR_TUNE_FORCE_OCC, int(tuned.get("occ", 0)))
        scgr.scgr_set_tuning(ctx, scgr.SCGR_TUNE_FORCE_RSQRT, int(tuned.get("rsqrt", 0)))
        scgr.scgr_set_tuning(ctx, scgr.SCGR_TUNE_FORCE_EX2POLY, int(tuned.get("ex2poly", 0)))


def bench_g_equals_s(args, scgr, torch, dev, Xd, Yd, tuned, peak_basis):
    """The g = s weighting of Sec. IV (every pair weighted by the similarity
    alone, without the aX aY factor of Eq. 10) on the 1M x 1M workload, p = 2,
    50 iterations: one whole registration (descriptors included) after a
    short warm-up, with the force kernel timed by CUDA events on the
    library's stream.  Per pair the counting convention drops the x aX flop:
    21 flops."""
    n, m = int(Xd.shape[0]), int(Yd.shape[0])
    stream = torch.cuda.current_stream()
    ctx = scgr.scgr_create(scgr.scgr_default_params(p=2.0, g_mode=0, k=16), stream)
    try:
        apply_plan(scgr, ctx, tuned)

        def one(iters):
            scgr.scgr_set_reference(ctx, Xd)
            scgr.scgr_set_template(ctx, Yd)
            scgr.scgr_compute_descriptors(ctx)
            scgr.scgr_run(ctx, iters)
            return scgr.scgr_get_result(ctx)

        one(2)
        torch.cuda.synchronize()
        scgr.scgr_set_force_timing(ctx, True)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        res = one(50)
        e1.record(stream)
        torch.cuda.synchronize()
        nforce, force_ms = scgr.scgr_get_force_timing(ctx)
        scgr.scgr_set_force_timing(ctx, False)
        plan = scgr.scgr_get_plan(ctx)
    finally:
        scgr.scgr_destroy(ctx)
    reg_ms = e0.elapsed_time(e1)
    avg = force_ms / max(nforce, 1)
    achieved = 21 * n * m / (avg * 1e-3) / 1e12
    peak, basis = peak_basis
    return {"workload": f"{n:,} x {m:,}, g = s (Sec. IV), p = 2, k = 16, 50 iterations",
            "ms_per_registration": reg_ms, "ms_per_iteration": reg_ms / 50,
            "pair_interactions_per_s": n * m * 50 / (reg_ms * 1e-3), "plan": plan, "scale": res.s,
            "roofline": {"bound": "alu", "kernel": "force_tile_kernel", "flops_per_pair": 21,
                         "force_launch_ms": avg, "force_launches_timed": nforce, "achieved": achieved,
                         "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak, "peak_basis": basis},
            "timing": "CUDA events on the library stream around one registration; force launches by the library's "
                      "own events"}


def bench_radius_registration(scgr, torch, dev, steps):
    """A whole registration with the radius neighbourhood of Sec. IV (radius
    sqrt(e) of each cloud's covariance) on the 35,000 x 30,800 case: both
    clouds' descriptors by the O(n^2) radius pass, then 200 iterations in a
    CUDA graph."""
    from paper_1902_01061_gb300 import synth
    sc = synth.scale_case()
    X = torch.from_numpy(sc.X).to(dev)
    Y = torch.from_numpy(sc.Y0).to(dev)
    ctx = scgr.scgr_create(scgr.scgr_default_params(p=2.0, neigh_mode=1, radius_scale=1.0, use_graph=1),
                           torch.cuda.current_stream())
    try:
        def one():
            scgr.scgr_set_reference(ctx, X)
            scgr.scgr_set_template(ctx, Y)
            scgr.scgr_compute_descriptors(ctx)
            scgr.scgr_run(ctx, 200)
            return scgr.scgr_get_result(ctx)
        sec = _timed(one, max(1, min(steps, 3)), 1, torch)
    finally:
        scgr.scgr_destroy(ctx)
    return {"workload": "35,000 x 30,800 points, radius neighbourhood sqrt(e) (scale 1.0), p=2, 200 iterations, "
                        "CUDA graph", "ms_per_registration": sec * 1e3,
            "timing": "host wall clock around synchronised calls"}


def bench_tiny(scgr, torch, dev, steps):
    """The 1,000 x 1,000 case (3-ellipsoid surface, 50 deg about x, p = 2,
    100 iterations): the latency regime, where the per-iteration launches and
    the float64 pose update dominate.  Whole registrations (descriptors +
    100 iterations) and the iterations alone, with the loop replayed from a
    CUDA graph and with eager launches."""
    from paper_1902_01061_gb300 import synth
    case = synth.tiny()
    X = torch.from_numpy(case.X).to(dev)
    Y = torch.from_numpy(case.Y0).to(dev)
    out = {"workload": "1,000 x 1,000 points, 50 deg about x, p=2, k=16, 100 iterations"}
    reps = max(5, min(steps, 20))
    for use_graph in (1, 0):
        ctx = scgr.scgr_create(scgr.scgr_default_params(p=2.0, use_graph=use_graph), torch.cuda.current_stream())
        try:
            def whole():
                scgr.scgr_set_reference(ctx, X)
                scgr.scgr_set_template(ctx, Y)
                scgr.scgr_compute_descriptors(ctx)
                scgr.scgr_run(ctx, 100)
                scgr.scgr_get_result(ctx)
            reg = _timed(whole, reps, 2, torch)

            def iters_only():
                scgr.scgr_set_state(ctx, state0)
                scgr.scgr_run(ctx, 100)
                scgr.scgr_get_result(ctx)
            scgr.scgr_set_reference(ctx, X)
            scgr.scgr_set_template(ctx, Y)
            scgr.scgr_compute_descriptors(ctx)
            state0 = scgr.scgr_get_state(ctx)
            it = _timed(iters_only, reps, 2, torch)
        finally:
            scgr.scgr_destroy(ctx)
        key = "graph" if use_graph else "eager"
        out[key] = {"ms_per_registration": reg * 1e3, "ms_per_iteration": it * 1e3 / 100}
    out["graph_speedup_per_iteration"] = out["eager"]["ms_per_iteration"] / out["graph"]["ms_per_iteration"]
    out["timing"] = "host wall clock around synchronised calls, mean of repeated runs"
    return out


def run_reference(args, ws, rank):
    """The oracle arm: bounded samples of the same workload on the host cores."""
    if rank != 0:
        return 0
    import numpy as np
    import oracle as O
    wl = WORKLOADS[args.workload]
    pair = make_pair(args.workload)
    n, m = len(pair.X), len(pair.Y0)
    rng = np.random.default_rng(77)
    aX = np.clip(rng.gamma(1.2, 0.015, size=n), 0, 0.33)
    aY = np.clip(rng.gamma(1.2, 0.015, size=m), 0, 0.33)
    sigma = O.sigma_auto(aX)
    Y = pair.Y0.astype(np.float64)
    rows_per_step = max(1, min(m, int(args.ref_rows)))
    def step():
        rows = np.sort(rng.choice(m, size=rows_per_step, replace=False))
        O.forces_rows(Y, pair.X, aY, aX, sigma, 2.0, 1, rows)
    for _ in range(args.warmup):
        step()
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        step()
        times.append(time.perf_counter() - t0)
    mean = sum(times) / len(times)
    value = rows_per_step * n / mean
    line = {
        "impl": "reference", "metric": metric_name(args.workload), "value": value, "unit": "pair-interactions/s",
        "n_gpus": ws, "steps": args.steps, "warmup": args.warmup, "ms_per_step": mean * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": base_config(args.workload, n, m),
        "cpu_baseline": {"value": value, "unit": "pair-interactions/s", "cores": 1, "kind": "oracle",
                         "sample": f"each step: iteration-0 force pass of {rows_per_step} random template rows "
                                   f"x {n} reference points, float64 numpy, single thread"},
        "e2e": {"value": value, "unit": "pair-interactions/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=list(WORKLOADS), default="large")
    ap.add_argument("--e2e-steps", type=int, default=None)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--ref-rows", type=int, default=48)
    ap.add_argument("--no-batch", action="store_true", help="skip the batched, differentiation and 35k legs")
    ap.add_argument("--no-autotune", action="store_true", help="keep the default tile shapes")
    ap.add_argument("--diff-only", action="store_true",
                    help="run only the differentiation leg (potential, recomputing and stored adjoints) and print it")
    ap.add_argument("--diff-n", type=int, default=50_000, help="points per cloud of the differentiation leg")
    ap.add_argument("--batch-only", action="store_true",
                    help="run only the batched leg (no one-call-per-pair comparison) and print it")
    ap.add_argument("--batch-iters", type=int, default=100, help="iterations of the batched leg")
    ap.add_argument("--next-only", action="store_true",
                    help="only the leg of the widened rows (odd-p fast path, radius, pyramid, change mask)")
    ap.add_argument("--split", choices=["none", "rows", "replicas"], default=None,
                    help="multi-GPU form: rows (default when WORLD_SIZE > 1) splits one registration by template rows "
                         "over the ranks; replicas runs the whole workload on every rank; none (default on one GPU) "
                         "is the single-context run")
    ap.add_argument("--p", type=float, default=2.0,
                    help="distance exponent of the main leg (default 2, the benchmark workload; 1 and 3 run the "
                         "odd-p fast paths, for profiling them)")
    ap.add_argument("--oracle-only", action="store_true",
                    help="only the oracle's timings on the host (sampled 1M x 1M force rows, configs 1 and 2)")
    ap.add_argument("--batch-plan", default=None, help="pin the batched force kernel 'P,CHUNK_TILES[,PERSISTENT]' (no autotuning)")
    ap.add_argument("--batch-eager", action="store_true", help="batched leg without the CUDA graph (for profilers)")
    ap.add_argument("--plan", default=None, help="pin the force kernel 'P,TPB[,OCC[,RSQRT[,EX2POLY]]]' (no autotuning), e.g. 4,128,2,0,1")
    args = ap.parse_args()
    ws, rank, local = dist_env()
    if args.impl == "reference":
        return run_reference(args, ws, rank)
    if args.oracle_only:
        if rank == 0:
            print(json.dumps({"leg": "oracle", "oracle_runs": oracle_runs(),
                              "sampled": cpu_baseline(make_pair(args.workload), 2.0, 1)}), flush=True)
        return 0

    import numpy as np
    import torch
    import torch.distributed as dist
    from paper_1902_01061_gb300 import scgr

    if not torch.cuda.is_available():
        raise RuntimeError("bench.py needs a CUDA GPU")
    torch.cuda.set_device(local)
    if ws > 1:
        dist.init_process_group("nccl")
    scgr.load()                      # fails loudly if the CUDA library is missing
    if args.batch_only:
        if rank == 0:
            out = bench_batch(args, scgr, torch, torch.device("cuda", local), args.steps, args.warmup)
            print(json.dumps({"leg": "batch", "steps": args.steps, "warmup": args.warmup, **out}), flush=True)
        return 0
    if args.diff_only:
        if rank == 0:
            out = bench_diff(args, scgr, torch, torch.device("cuda", local), args.steps, args.warmup)
            print(json.dumps({"leg": "differentiation", "steps": args.steps, "warmup": args.warmup, **out}),
                  flush=True)
        return 0
    if args.next_only:
        if rank == 0:
            dev = torch.device("cuda", local)
            pair = make_pair(args.workload)
            Xd, Yd = torch.from_numpy(pair.X).to(dev), torch.from_numpy(pair.Y0).to(dev)
            out = bench_next(args, scgr, torch, dev, args.steps, args.warmup, Xd, Yd)
            nsm = torch.cuda.get_device_properties(dev).multi_processor_count
            peak = (2 * FP32_LANES_PER_SM * nsm * 2070e6 / 1e12,
                    f"2 x {FP32_LANES_PER_SM} FP32 lanes x {nsm} SMs x 2070 MHz (max clock)")
            out["g_equals_s_full_size"] = bench_g_equals_s(args, scgr, torch, dev, Xd, Yd, None, peak)
            out["radius_registration"] = bench_radius_registration(scgr, torch, dev, args.steps)
            out["tiny_case"] = bench_tiny(scgr, torch, dev, args.steps)
            print(json.dumps({"leg": "next_rows", "steps": args.steps, **out}), flush=True)
        return 0
    wl = WORKLOADS[args.workload]
    pair = make_pair(args.workload)
    n, m, iters = len(pair.X), len(pair.Y0), wl["iters"]
    pairs_per_step = n * m * iters
    dev = torch.device("cuda", local)
    Xd = torch.from_numpy(pair.X).to(dev)
    Yd = torch.from_numpy(pair.Y0).to(dev)
    moved = torch.empty((m, 3), dtype=torch.float32, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    split = args.split or ("rows" if ws > 1 else "none")
    rows_mode = split == "rows"
    from paper_1902_01061_gb300 import shard
    row0, nrows = shard.row_partition(m, ws, rank) if rows_mode else (0, m)
    # row sharding iterates stepwise, which needs the Eq. 12 horizon up front
    params = scgr.scgr_default_params(p=args.p, g_mode=1, k=16, E=iters if rows_mode else 0)
    stream = torch.cuda.current_stream()
    ctx = scgr.scgr_create(params, stream)
    num_sms = torch.cuda.get_device_properties(dev).multi_processor_count
    part_buf = torch.empty(13, dtype=torch.float64, device=dev)
    Xh = torch.from_numpy(pair.X).pin_memory().numpy()      # pinned host copies for the end-to-end leg
    Yh = torch.from_numpy(pair.Y0).pin_memory().numpy()

    def load_clouds(host=False):
        if host:
            scgr.scgr_set_reference_host(ctx, Xh)
            scgr.scgr_set_template_host(ctx, Yh)
        else:
            scgr.scgr_set_reference(ctx, Xd)
            scgr.scgr_set_template(ctx, Yd)
        if rows_mode:
            scgr.scgr_set_row_range(ctx, row0, nrows)
        scgr.scgr_compute_descriptors(ctx)

    def iterate():
        if not rows_mode:
            scgr.scgr_run(ctx, iters)
            return
        # this rank's template rows; the 13 partial sums all-gathered on the
        # device (NCCL) and added in rank order by the library each iteration
        for _ in range(iters):
            scgr.scgr_step_partials_dev(ctx, part_buf)
            scgr.scgr_step_apply_dev(ctx, shard.gather_parts(part_buf))

    tuned = None
    if args.plan:
        vals = [int(v) for v in args.plan.split(",")]
        P_, T_, O_ = vals[0], vals[1], (vals[2] if len(vals) > 2 else 0)
        R_ = vals[3] if len(vals) > 3 else 0
        E_ = vals[4] if len(vals) > 4 else 0
        scgr.scgr_set_tuning(ctx, scgr.SCGR_TUNE_FORCE_P, P_)
        scgr.scgr_set_tuning(ctx, scgr.SCGR_TUNE_FORCE_TPB, T_)
        scgr.scgr_set_tuning(ctx, scgr.SCGR_TUNE_FORCE_OCC, O_)
        scgr.scgr_set_tuning(ctx, scgr.SCGR_TUNE_FORCE_RSQRT, R_)
        scgr.scgr_set_tuning(ctx, scgr.SCGR_TUNE_FORCE_EX2POLY, E_)
        tuned = {"P": P_, "tpb": T_, "occ": O_, "rsqrt": R_, "ex2poly": E_, "pinned": True}
    elif not args.no_autotune:
        from paper_1902_01061_gb300 import autotune
        load_clouds()
        tuned = autotune.tune_single(ctx, n, nrows, args.p, reps=2)

    def step_device():
        load_clouds()
        iterate()
        scgr.scgr_get_moved(ctx, moved)

    for _ in range(args.warmup):
        step_device()
        scgr.scgr_get_result(ctx)
    torch.cuda.synchronize()

    clocks = ClockSampler(gpu_index_for(local))
    scgr.scgr_set_force_timing(ctx, True)
    launches0 = scgr.scgr_launch_count(ctx)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    wall0 = time.perf_counter()
    for k in range(args.steps):
        flush.zero_()                # evict L2 between steps (outside the events)
        ev[k][0].record(stream)
        step_device()
        ev[k][1].record(stream)
    torch.cuda.synchronize()
    wall = time.perf_counter() - wall0
    clk = clocks.stop()
    if ws > 1:
        dist.barrier()
    res = scgr.scgr_get_result(ctx)
    launches = scgr.scgr_launch_count(ctx) - launches0
    nforce, force_ms = scgr.scgr_get_force_timing(ctx)
    scgr.scgr_set_force_timing(ctx, False)
    step_ms = [a.elapsed_time(b) for a, b in ev]
    ms_per_step = sum(step_ms) / len(step_ms)
    if ws > 1:
        t = torch.tensor([ms_per_step], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms_per_step = float(t.item())
    # replicas: every rank registers the whole workload (weak scaling);
    # rows: the ranks share one registration (strong scaling)
    units = pairs_per_step if rows_mode else ws * pairs_per_step
    value = units / (ms_per_step * 1e-3)
    force_avg_ms = force_ms / max(nforce, 1)

    # end to end through the host entry points (pinned host buffers)
    e2e_steps = args.e2e_steps if args.e2e_steps is not None else min(args.steps, 3)
    e2e = None
    if e2e_steps > 0:
        Mh = torch.empty((m, 3), dtype=torch.float32).pin_memory().numpy()
        times = []
        for _ in range(e2e_steps):
            flush.zero_()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            load_clouds(host=True)
            iterate()
            scgr.scgr_get_moved_host(ctx, Mh)
            scgr.scgr_get_result(ctx)
            times.append(time.perf_counter() - t0)
        e2e_s = sum(times) / len(times)
        if ws > 1:
            t = torch.tensor([e2e_s], device=dev)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            e2e_s = float(t.item())
        e2e = {"value": units / e2e_s, "unit": "pair-interactions/s",
               "h2d_bytes_per_step": (n + m) * 12, "d2h_bytes_per_step": m * 12 + 8 * 13 + 8}
    scgr.scgr_destroy(ctx)
    sm_max_mhz = (clk or {}).get("sm_max_mhz") or 2070.0
    sm_mhz = (clk or {}).get("sm_mhz")
    peak_tflops = 2 * FP32_LANES_PER_SM * num_sms * sm_max_mhz * 1e6 / 1e12
    peak_basis = f"2 x {FP32_LANES_PER_SM} FP32 lanes x {num_sms} SMs x {sm_max_mhz:.0f} MHz (max clock)"
    batch = diff = scale = nxt = tiny = None
    if ws == 1 and not args.no_batch:
        batch = bench_batch(args, scgr, torch, dev, args.steps, args.warmup)
        diff = bench_diff(args, scgr, torch, dev, args.steps, args.warmup)
        scale = bench_scale(args, scgr, torch, dev, args.steps, args.warmup)
        tiny = bench_tiny(scgr, torch, dev, args.steps)
        nxt = bench_next(args, scgr, torch, dev, args.steps, args.warmup, Xd, Yd)
        nxt["g_equals_s_full_size"] = bench_g_equals_s(args, scgr, torch, dev, Xd, Yd, tuned,
                                                       (peak_tflops, peak_basis))
        nxt["radius_registration"] = bench_radius_registration(scgr, torch, dev, args.steps)

    if rank != 0:
        if ws > 1:
            dist.destroy_process_group()
        return 0

    traffic, digest = profile_traffic()
    if nforce > 0:
        achieved_tflops = FLOPS_PER_PAIR * n * nrows / (force_avg_ms * 1e-3) / 1e12   # one launch: this rank's rows
        roofline = {"bound": "alu", "achieved": achieved_tflops, "peak": peak_tflops, "unit": "TFLOP/s",
                    "frac": achieved_tflops / peak_tflops, "traffic": traffic,
                    "kernel": "force_tile_kernel", "flops_per_pair": FLOPS_PER_PAIR,
                    "force_launch_ms": force_avg_ms, "force_launches_timed": nforce,
                    "peak_basis": peak_basis}
        if sm_mhz:
            roofline["frac_at_measured_clock"] = achieved_tflops / (peak_tflops * sm_mhz / sm_max_mhz)
    else:
        # the odd-p fast paths (--p 1 after its first pass, --p 3 always) launch no all-pairs force kernel
        roofline = {"bound": "alu", "achieved": None, "peak": peak_tflops, "unit": "TFLOP/s", "frac": None,
                    "traffic": None, "kernel": "force_tile_kernel", "force_launches_timed": 0,
                    "peak_basis": peak_basis}
    line = {
        "metric": metric_name(args.workload),
        "value": value, "unit": "pair-interactions/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
        "scaling": "strong" if rows_mode else "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "ms_per_iteration": ms_per_step / iters,
        "pct_fp32_peak": 100.0 * roofline["frac"] if roofline["frac"] is not None else None,
        "config": dict(base_config(args.workload, n, m), p=args.p, autotuned=tuned,
                       l2="flushed between steps (256 MB write)",
                       parallelism=(f"rows x{ws} (template rows split over the ranks, 13 float64 partial sums "
                                    f"all-gathered on the device per iteration)" if rows_mode else f"replicas x{ws}")),
        "gpu_launches": launches,
        "wall_s_timed_region": wall,
        "pose": {"s": res.s, "iterations": res.iterations},
        "clocks": clk,
        "roofline": roofline,
        "e2e": e2e,
        "batch": batch,
        "differentiation": diff,
        "scale_case": scale,
        "tiny_case": tiny,
        "next_rows": nxt,
    }
    line["peaks_measured"] = measured_peaks(scgr, num_sms, sm_mhz or sm_max_mhz)
    # the co-bound of the p = 2 force kernel: one ex2 and one sqrt per pair on
    # the special-function unit, at the rates just measured
    pk = line["peaks_measured"]
    sfu = 1.0 / (1.0 / pk["mufu_ex2"]["per_clk_per_sm"] + 1.0 / pk["mufu_sqrt"]["per_clk_per_sm"])
    clk_mhz = sm_mhz or sm_max_mhz
    if nforce > 0:
        got = n * nrows / (force_avg_ms * 1e-3) / (num_sms * clk_mhz * 1e6)
        roofline["pairs_per_clk_per_sm"] = got
        roofline["sfu_bound_pairs_per_clk_per_sm"] = sfu
        roofline["frac_of_sfu_bound"] = got / sfu
    if ws == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(pair, 2.0, 1)
        try:
            line["cpu_baseline"]["oracle_runs"] = oracle_runs()
        except Exception as e:                   # the sampled figure stands on its own
            line["cpu_baseline"]["oracle_runs"] = {"unavailable": f"{type(e).__name__}: {e}"[:200]}
    print(json.dumps(line), flush=True)
    if ws > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
