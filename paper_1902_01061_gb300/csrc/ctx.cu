// Internal helpers of the C ABI: argument checks, buffers, error words, the
// descriptor pass and the iteration launch sequence.
#include <cuda_runtime.h>

#include <atomic>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "context.cuh"

using namespace scgr;

namespace scgr {
namespace api {

scgr_status fail(scgr_ctx* c, scgr_status st, const std::string& msg) {
  if (c) c->err = msg;
  return st;
}

scgr_status cuda_fail(scgr_ctx* c, cudaError_t e, const char* where) {
  cudaGetLastError();  // clear a sticky launch error where possible
  std::string msg = std::string(where) + ": " + cudaGetErrorString(e);
  if (e == cudaErrorMemoryAllocation) return fail(c, SCGR_ERR_OOM, msg);
  return fail(c, SCGR_ERR_CUDA, msg);
}

// Test hook: while > 0, the next allocations fail (host-side fault
// injection; nothing is asked of the device).
std::atomic<int> g_fail_allocs{0};

cudaError_t ensure(DevBuf& b, size_t bytes) {
  if (bytes == 0) bytes = 16;
  if (b.cap >= bytes) return cudaSuccess;
  if (g_fail_allocs.load() > 0) {
    g_fail_allocs.fetch_sub(1);
    return cudaErrorMemoryAllocation;
  }
  if (b.p) cudaFree(b.p);
  b.p = nullptr;
  b.cap = 0;
  cudaError_t e = cudaMalloc(&b.p, bytes);
  if (e == cudaSuccess) b.cap = bytes;
  return e;
}

void release(DevBuf& b) {
  if (b.p) cudaFree(b.p);
  b.p = nullptr;
  b.cap = 0;
}

scgr_status check_params(const scgr_params* p, std::string& why) {
  if (!p) { why = "params is NULL"; return SCGR_ERR_INVALID_ARG; }
  if (p->k < 3 || p->k > 32) { why = "k must be in [3, 32]"; return SCGR_ERR_INVALID_ARG; }
  if (!(p->p >= 1.0) || !std::isfinite(p->p)) { why = "p must be finite and >= 1 (Eq. 11)"; return SCGR_ERR_INVALID_ARG; }
  if (!std::isfinite(p->sigma)) { why = "sigma must be finite"; return SCGR_ERR_INVALID_ARG; }
  if (p->g_mode != 0 && p->g_mode != 1) { why = "g_mode must be 0 or 1"; return SCGR_ERR_INVALID_ARG; }
  if (!(p->G1 > 0.0) || !std::isfinite(p->G1)) { why = "G1 must be > 0"; return SCGR_ERR_INVALID_ARG; }
  if (p->step_mode != 0 && p->step_mode != 1) { why = "step_mode must be 0 or 1"; return SCGR_ERR_INVALID_ARG; }
  if (!(p->eta0 > 0.0) || !std::isfinite(p->eta0)) { why = "eta0 must be > 0"; return SCGR_ERR_INVALID_ARG; }
  if (!std::isfinite(p->time)) { why = "time must be finite"; return SCGR_ERR_INVALID_ARG; }
  if (p->scale_mode < 0 || p->scale_mode > 2) { why = "scale_mode must be 0, 1 or 2"; return SCGR_ERR_INVALID_ARG; }
  if (p->neigh_mode != 0 && p->neigh_mode != 1) { why = "neigh_mode must be 0 or 1"; return SCGR_ERR_INVALID_ARG; }
  if (p->neigh_mode == 1 && !(p->radius_scale > 0.0 && std::isfinite(p->radius_scale))) { why = "radius_scale must be > 0"; return SCGR_ERR_INVALID_ARG; }
  return SCGR_OK;
}

StepParams step_params(const scgr_ctx* c) {
  StepParams sp;
  sp.G1 = c->prm.G1;
  sp.eta0 = c->prm.eta0;
  sp.time = c->prm.time;
  sp.step_mode = c->prm.step_mode;
  sp.scale_mode = c->prm.scale_mode;
  sp.M = (int)c->m;
  return sp;
}

scgr_status read_error_word(scgr_ctx* c) {
  int h = 0;
  SCGR_CK(c, cudaMemcpyAsync(&h, c->errword, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  SCGR_CK(c, cudaStreamSynchronize(c->stream));
  if (h == 0) return SCGR_OK;
  SCGR_CK(c, cudaMemsetAsync(c->errword, 0, sizeof(int), c->stream));
  SCGR_CK(c, cudaStreamSynchronize(c->stream));
  if (h & ERR_NONFINITE)
    return fail(c, SCGR_ERR_NONFINITE, "an input coordinate is NaN/Inf or larger than 1e18 in magnitude");
  if (h & ERR_TIMEOUT) return fail(c, SCGR_ERR_TIMEOUT, "a bounded device-side wait gave up");
  return fail(c, SCGR_ERR_NUMERIC, "the iteration step became non-finite (zero or non-finite total weight)");
}

scgr_status set_cloud(scgr_ctx* c, const float* xyz, int64_t n, bool host, bool ref) {
  if (!c) return SCGR_ERR_INVALID_ARG;
  c->err.clear();
  if (!xyz) return fail(c, SCGR_ERR_INVALID_ARG, "xyz is NULL");
  const int64_t minpts = ref ? c->prm.k : (c->prm.k > 3 ? c->prm.k : 3);
  if (n < minpts) return fail(c, SCGR_ERR_INVALID_ARG, ref ? "reference has fewer than k points" : "template has fewer than max(k, 3) points");
  if (n > (int64_t(1) << 30)) return fail(c, SCGR_ERR_INVALID_ARG, "more than 2^30 points");
  DevBuf& dst = ref ? c->X4 : c->Y4;
  SCGR_CK(c, ensure(dst, (size_t)n * sizeof(float4)));
  const float* src = xyz;
  if (host) {
    SCGR_CK(c, ensure(c->stage, (size_t)n * 3 * sizeof(float)));
    SCGR_CK(c, cudaMemcpyAsync(c->stage.p, xyz, (size_t)n * 3 * sizeof(float), cudaMemcpyHostToDevice, c->stream));
    src = (const float*)c->stage.p;
  }
  SCGR_CK(c, launch_pack(c->L(), src, n, (float4*)dst.p, c->errword));
  if (ref) { c->n = n; c->have_X = true; c->rgrid_ok = false; }
  else { c->m = n; c->have_Y = true; }
  c->have_desc = false;
  return SCGR_OK;
}

// Launch the force kernel, bracketed by timing events when enabled.
scgr_status force_launch(scgr_ctx* c) {
  const int ntiles = (int)(c->npad / c->fp.tile_j);
  const bool timed = c->timing && !c->capturing;
  if (timed) {
    if (c->ev_used + 2 > c->ev.size()) {
      for (int q = 0; q < 2; ++q) {
        cudaEvent_t e;
        SCGR_CK(c, cudaEventCreate(&e));
        c->ev.push_back(e);
      }
    }
    SCGR_CK(c, cudaEventRecord(c->ev[c->ev_used], c->stream));
  }
  SCGR_CK(c, launch_force(c->L(), c->fp, (const float4*)c->Xr.p, (const float2*)c->XA.p, ntiles,
                          (const float4*)c->Y0r.p, (int)c->mpad, c->pose, c->qexp, (float4*)c->partial.p));
  if (timed) {
    SCGR_CK(c, cudaEventRecord(c->ev[c->ev_used + 1], c->stream));
    c->ev_used += 2;
  }
  return SCGR_OK;
}

// Fold finished event pairs into the tally (the stream must be idle).
scgr_status collect_timing(scgr_ctx* c) {
  for (size_t q = 0; q + 1 < c->ev_used; q += 2) {
    float ms = 0.f;
    SCGR_CK(c, cudaEventElapsedTime(&ms, c->ev[q], c->ev[q + 1]));
    c->timed_ms += ms;
    c->timed_launches += 1;
  }
  c->ev_used = 0;
  return SCGR_OK;
}

// Grid spec of a cloud and the workspace of its grid (one host
// synchronisation for the bounding box).
static scgr_status grid_setup(scgr_ctx* c, const float4* P, int n, GridSpec* gs_out) {
  SCGR_CK(c, ensure(c->gbb, sizeof(float) * (256 * 6 + 8)));
  float* part = (float*)c->gbb.p;
  SCGR_CK(c, launch_bbox(c->L(), P, n, part, part + 256 * 6));
  float bb[6];
  SCGR_CK(c, cudaMemcpyAsync(bb, part + 256 * 6, sizeof(bb), cudaMemcpyDeviceToHost, c->stream));
  SCGR_CK(c, cudaStreamSynchronize(c->stream));
  const GridSpec gs = make_grid_spec(bb, n);
  const int64_t ncell = grid_cells(gs);
  SCGR_CK(c, ensure(c->gcell, (size_t)n * sizeof(int)));
  SCGR_CK(c, ensure(c->gcount, (size_t)ncell * sizeof(int)));
  SCGR_CK(c, ensure(c->gcursor, (size_t)ncell * sizeof(int)));
  SCGR_CK(c, ensure(c->gstart, (size_t)(ncell + 1) * sizeof(int)));
  SCGR_CK(c, ensure(c->gblock, (size_t)((ncell + 1023) / 1024 + 1) * sizeof(int)));
  SCGR_CK(c, ensure(c->gsorted, (size_t)n * sizeof(float4)));
  SCGR_CK(c, ensure(c->gsidx, (size_t)n * sizeof(int)));
  *gs_out = gs;
  return SCGR_OK;
}

// k nearest neighbours of one cloud: brute force below knn_grid_min points,
// the exact grid search above.
scgr_status knn_cloud(scgr_ctx* c, const float4* P, int n, int32_t* out) {
  const int k = c->prm.k;
  if ((int64_t)n < c->knn_grid_min) {
    SCGR_CK(c, launch_knn(c->L(), P, n, k, out));
    return SCGR_OK;
  }
  GridSpec gs;
  const scgr_status st = grid_setup(c, P, n, &gs);
  if (st != SCGR_OK) return st;
  SCGR_CK(c, launch_knn_grid(c->L(), P, n, k, gs, (int*)c->gcell.p, (int*)c->gcount.p, (int*)c->gstart.p,
                             (int*)c->gcursor.p, (int*)c->gblock.p, (float4*)c->gsorted.p, (int*)c->gsidx.p, out));
  return SCGR_OK;
}

// Nearest reference point of nq external queries (float32 [nq][3] on the
// device): brute force below nearest_grid_min reference points, else the exact
// two-level grid search over the reference (the same result): fine cells
// around the query, then coarse cells that skip empty space.  The
// reference's two grids are built on the first query after
// scgr_set_reference and kept in their own buffers (the descriptor pass
// reuses the shared grid workspace for both clouds), so later queries skip
// the bounding-box synchronisation and the counting sorts.
scgr_status nearest_reference(scgr_ctx* c, const float* q3, int nq, int32_t* idx_out, float* key_out) {
  const float4* X4 = (const float4*)c->X4.p;
  const int n = (int)c->n;
  if ((int64_t)n < c->nearest_grid_min) {
    SCGR_CK(c, launch_nearest(c->L(), X4, n, q3, nq, idx_out, key_out));
    return SCGR_OK;
  }
  if (!c->rgrid_ok) {
    GridSpec gs;
    const scgr_status st = grid_setup(c, X4, n, &gs);
    if (st != SCGR_OK) return st;
    const int64_t ncell = grid_cells(gs);
    SCGR_CK(c, ensure(c->rgstart, (size_t)(ncell + 1) * sizeof(int)));
    SCGR_CK(c, ensure(c->rgsorted, (size_t)n * sizeof(float4)));
    SCGR_CK(c, ensure(c->rgsidx, (size_t)n * sizeof(int)));
    SCGR_CK(c, launch_grid_build(c->L(), X4, n, gs, (int*)c->gcell.p, (int*)c->gcount.p, (int*)c->rgstart.p,
                                 (int*)c->gcursor.p, (int*)c->gblock.p, (float4*)c->rgsorted.p, (int*)c->rgsidx.p));
    // the coarse level: the same counting sort with cells NEAREST_COARSE times larger
    // (it fits the fine level's count/cursor/block scratch)
    const GridSpec gc = coarse_grid_spec(gs);
    SCGR_CK(c, ensure(c->rcgstart, (size_t)(grid_cells(gc) + 1) * sizeof(int)));
    SCGR_CK(c, ensure(c->rcgsorted, (size_t)n * sizeof(float4)));
    SCGR_CK(c, ensure(c->rcgsidx, (size_t)n * sizeof(int)));
    SCGR_CK(c, launch_grid_build(c->L(), X4, n, gc, (int*)c->gcell.p, (int*)c->gcount.p, (int*)c->rcgstart.p,
                                 (int*)c->gcursor.p, (int*)c->gblock.p, (float4*)c->rcgsorted.p, (int*)c->rcgsidx.p));
    c->rgspec = gs;
    c->rcgspec = gc;
    c->rgrid_ok = true;
  }
  if (c->nearest_levels == 1) {
    SCGR_CK(c, launch_nearest_grid(c->L(), (const float4*)c->rgsorted.p, (const int*)c->rgsidx.p,
                                   (const int*)c->rgstart.p, c->rgspec, q3, nq, idx_out, key_out));
  } else {
    SCGR_CK(c, launch_nearest_grid2(c->L(), (const float4*)c->rgsorted.p, (const int*)c->rgsidx.p,
                                    (const int*)c->rgstart.p, c->rgspec, (const float4*)c->rcgsorted.p,
                                    (const int*)c->rcgsidx.p, (const int*)c->rcgstart.p, c->rcgspec, q3, nq, idx_out,
                                    key_out));
  }
  return SCGR_OK;
}

// Curvature of both clouds for the current neighbourhood mode (k nearest or
// radius), then sigma (scaled by sigma_scale).
scgr_status curvatures(scgr_ctx* c, int k, double radius_scale, double sigma_scale) {
  const int n = (int)c->n, m = (int)c->m;
  Launch L = c->L();
  const float4* X4 = (const float4*)c->X4.p;
  const float4* Y4 = (const float4*)c->Y4.p;
  DevStats* st = c->stats;
  if (c->prm.neigh_mode == 0) {
    SCGR_CK(c, ensure(c->knnX, (size_t)n * k * sizeof(int32_t)));
    SCGR_CK(c, ensure(c->knnY, (size_t)m * k * sizeof(int32_t)));
    const int k_prev = c->prm.k;
    c->prm.k = k;
    scgr_status ks = knn_cloud(c, X4, n, (int32_t*)c->knnX.p);
    if (ks == SCGR_OK) ks = knn_cloud(c, Y4, m, (int32_t*)c->knnY.p);
    if (ks != SCGR_OK) {
      c->prm.k = k_prev;
      return ks;
    }
    SCGR_CK(c, launch_curvature(L, X4, (const int32_t*)c->knnX.p, n, k, (double*)c->aX64.p, (float*)c->aX32.p));
    SCGR_CK(c, launch_curvature(L, Y4, (const int32_t*)c->knnY.p, m, k, (double*)c->aY64.p, (float*)c->aY32.p));
  } else {
    c->prm.radius_scale = radius_scale;
    const double s2 = radius_scale * radius_scale;
    SCGR_CK(c, launch_radius_curvature(L, X4, n, &st->eX, s2, (double*)c->aX64.p, (float*)c->aX32.p, nullptr));
    SCGR_CK(c, launch_radius_curvature(L, Y4, m, &st->eY0, s2, (double*)c->aY64.p, (float*)c->aY32.p, nullptr));
  }
  const double user = c->prm.sigma > 0.0 ? c->prm.sigma * sigma_scale : 0.0;
  SCGR_CK(c, launch_sigma(L, (const double*)c->aX64.p, n, user, c->red, &st->sigma, &st->asum[0]));
  if (user <= 0.0 && sigma_scale != 1.0) SCGR_CK(c, launch_scale_double(L, &st->sigma, sigma_scale));
  return SCGR_OK;
}

// Recompute the force plan (after a tuning change) and the buffers and
// template records that depend on it; descriptors and pose are kept.
scgr_status replan(scgr_ctx* c) {
  const int64_t mloc = c->rows >= 0 ? c->rows : c->m;
  c->fp = plan_force(mloc, c->npad, c->prm.p, c->num_sms, c->ftune);
  c->mpad = force_mpad(mloc, c->fp);
  SCGR_CK(c, ensure(c->Y0r, (size_t)c->mpad * sizeof(float4)));
  SCGR_CK(c, ensure(c->partial, (size_t)c->fp.splits * c->mpad * sizeof(float4)));
  SCGR_CK(c, ensure(c->blockpart, (size_t)combine_blocks(c->mpad) * 13 * sizeof(double)));
  SCGR_CK(c, launch_records(c->L(), (const float4*)c->X4.p, (const double*)c->aX64.p, (int)c->n, (int)c->npad,
                            (const float4*)c->Y4.p + c->row0, (const double*)c->aY64.p + c->row0, (int)mloc,
                            (int)c->mpad, c->prm.g_mode, c->stats, (float4*)c->Xr.p, (float2*)c->XA.p,
                            (float4*)c->Y0r.p));
  drop_graph(c);
  return SCGR_OK;
}

// Odd integer p needs no all-pairs pass per iteration.  For p = 1 the pair
// weight aX s_ij d^0 does not depend on the pose, so the force kernel's
// per-split sums (sum w, sum w X') are the same in every iteration: the first
// iteration of a run computes them and the others reuse them (bit-identical).
// For p = 3 the sums are a quadratic form in the template point over 14
// pose-free moments of g (computed once per run; an exact re-association, so
// equal to the direct pass up to rounding).
scgr_status enqueue_iterations(scgr_ctx* c, int iters) {
  const int nb = combine_blocks(c->mpad);
  const StepParams sp = step_params(c);
  const bool pose_free = c->fp.pmode == 1 && c->reuse_pose_free;
  const bool moments = c->fp.pmode == 3 && c->reuse_pose_free;
  const int mloc = (int)(c->rows >= 0 ? c->rows : c->m);
  if (moments && iters > 0) {
    const int ntiles = (int)(c->npad / c->fp.tile_j);
    const int S = moments_splits(ntiles, c->num_sms, c->mpad);
    SCGR_CK(c, ensure(c->mpart, (size_t)S * c->mpad * 14 * sizeof(double)));
    SCGR_CK(c, ensure(c->mom, (size_t)c->mpad * 14 * sizeof(double)));
    SCGR_CK(c, launch_moments(c->L(), (const float4*)c->Xr.p, (const float2*)c->XA.p, ntiles, (const float4*)c->Y0r.p,
                              (int)c->mpad, mloc, S, (double*)c->mpart.p, (double*)c->mom.p));
  }
  for (int t = 0; t < iters; ++t) {
    if (moments) {
      SCGR_CK(c, launch_combine_moments(c->L(), (const double*)c->mom.p, mloc, (int)c->mpad, (const float4*)c->Y0r.p,
                                        (const double*)c->aY64.p, c->prm.g_mode, c->pose, nullptr,
                                        (double*)c->blockpart.p));
      SCGR_CK(c, launch_finalize(c->L(), (const double*)c->blockpart.p, nb, c->pose, c->stats, sp, c->errword));
      continue;
    }
    if (!(pose_free && t > 0)) {
      scgr_status fs = force_launch(c);
      if (fs != SCGR_OK) return fs;
    }
    if (c->fused_tail && c->mpad <= FUSED_MAX_SLOTS) {
      // small templates: combine and finalize in one block (one launch less per iteration)
      SCGR_CK(c, launch_combine_finalize(c->L(), (const float4*)c->partial.p, c->fp.splits, (int)c->mpad, (int)c->m,
                                         (const float4*)c->Y0r.p, (const float*)c->aY32.p, c->prm.g_mode, c->pose,
                                         c->stats, sp, c->errword));
      continue;
    }
    SCGR_CK(c, launch_combine(c->L(), (const float4*)c->partial.p, c->fp.splits, (int)c->mpad, (int)c->m,
                              (const float4*)c->Y0r.p, (const float*)c->aY32.p, c->prm.g_mode, c->pose,
                              nullptr, (double*)c->blockpart.p));
    SCGR_CK(c, launch_finalize(c->L(), (const double*)c->blockpart.p, nb, c->pose, c->stats, sp, c->errword));
  }
  return SCGR_OK;
}

void drop_graph(scgr_ctx* c) {
  if (c->gexec) cudaGraphExecDestroy(c->gexec);
  if (c->graph) cudaGraphDestroy(c->graph);
  c->gexec = nullptr;
  c->graph = nullptr;
  c->graph_iters = -1;
}

}  // namespace api
}  // namespace scgr
