// C ABI of the scgr library: context, buffers, argument checks and the
// launch sequence of the method (see include/scgr.h for the contract).
#include <cuda_runtime.h>

#include <climits>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <algorithm>
#include <string>
#include <vector>

#include "common.cuh"
#include "scgr.h"

using namespace scgr;

namespace {

struct DevBuf {
  void* p = nullptr;
  size_t cap = 0;
};

thread_local std::string g_create_error;

}  // namespace

struct scgr_ctx {
  scgr_params prm{};
  cudaStream_t stream = nullptr;
  int device = 0;
  int num_sms = 0;
  std::string err;
  int64_t n = 0, m = 0, npad = 0, mpad = 0;
  int64_t row0 = 0, rows = -1;  // template rows whose forces this context computes (rows < 0: all)
  bool have_X = false, have_Y = false, have_desc = false;
  int E_host = 0;          // Eq. 12 horizon in use (0: not fixed yet)
  int iterations = 0;      // iterations enqueued since the descriptors
  int64_t launches = 0;
  ForcePlan fp{};
  float qexp = 0.f;        // (p - 1) / 2, exponent of d^2 in the weight

  DevBuf X4, Y4, stage, knnX, knnY, aX64, aY64, aX32, aY32, Xr, XA, Y0r, partial, blockpart,
      moved_stage;
  DevPose* pose = nullptr;
  DevPose* pose_eval = nullptr;  // pose of a potential / gradient evaluation
  double* aux = nullptr;         // [0,13) forward sums, [16,29) adjoint sums, [32,39) grad7, [48,55) pose7
  DevStats* stats = nullptr;
  int* errword = nullptr;
  double* red = nullptr;   // reduction scratch

  cudaGraph_t graph = nullptr;
  cudaGraphExec_t gexec = nullptr;
  int graph_iters = -1;
  bool capturing = false;
  cudaStream_t cap_stream = nullptr;  // capture / replay stream (never the legacy stream)
  cudaEvent_t join_in = nullptr, join_out = nullptr;

  // batch workspace
  DevBuf bX4, bY4, bknnX, bknnY, baX64, baY64, baX32, baY32, bXr, bXA, bY0r, bpartial, bblockpart,
      bpairs, bitems, bcpair, btabX, btabY, bxoff, byoff, bstats, bposes;
  int batch_chunk_tiles = 16;   // reference tiles per batched work item (tunable)
  int batch_P = 1;              // template points per thread in the batched force kernel (tunable)
  int64_t knn_grid_min = 65536; // clouds with at least this many points use the grid kNN (tunable)
  ForceTuning ftune;            // force-plan overrides (tunable)
  int reuse_pose_free = 1;      // p = 1: one force pass per scgr_run (tunable)
  DevBuf gcell, gcount, gstart, gcursor, gblock, gsorted, gsidx, gbb, cd_key, cd_moved, wstore, wupart, wpartial,
      mpart, mom;
  cudaGraph_t bgraph = nullptr;
  cudaGraphExec_t bgexec = nullptr;

  // force-kernel timing (diagnostic)
  bool timing = false;
  std::vector<cudaEvent_t> ev;  // pairs (start, end)
  size_t ev_used = 0;
  double timed_ms = 0.0;
  int64_t timed_launches = 0;

  Launch L() { return Launch{stream, &launches}; }
};

namespace {

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

#define SCGR_CK(ctx, call)                                  \
  do {                                                      \
    cudaError_t e_ = (call);                                \
    if (e_ != cudaSuccess) return cuda_fail(ctx, e_, #call); \
  } while (0)

cudaError_t ensure(DevBuf& b, size_t bytes) {
  if (bytes == 0) bytes = 16;
  if (b.cap >= bytes) return cudaSuccess;
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
  if (ref) { c->n = n; c->have_X = true; }
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

// k nearest neighbours of one cloud: brute force below knn_grid_min points,
// the exact grid search above (one host synchronisation for the box).
scgr_status knn_cloud(scgr_ctx* c, const float4* P, int n, int32_t* out) {
  const int k = c->prm.k;
  if ((int64_t)n < c->knn_grid_min) {
    SCGR_CK(c, launch_knn(c->L(), P, n, k, out));
    return SCGR_OK;
  }
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
  SCGR_CK(c, launch_knn_grid(c->L(), P, n, k, gs, (int*)c->gcell.p, (int*)c->gcount.p, (int*)c->gstart.p,
                             (int*)c->gcursor.p, (int*)c->gblock.p, (float4*)c->gsorted.p, (int*)c->gsidx.p, out));
  return SCGR_OK;
}

void drop_graph(scgr_ctx* c);

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
    SCGR_CK(c, launch_combine(c->L(), (const float4*)c->partial.p, c->fp.splits, (int)c->mpad, (int)c->m,
                              (const float4*)c->Y0r.p, (const double*)c->aY64.p, c->prm.g_mode, c->pose,
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

}  // namespace

extern "C" {

scgr_status scgr_default_params(scgr_params* out) {
  if (!out) return SCGR_ERR_INVALID_ARG;
  std::memset(out, 0, sizeof(*out));
  out->k = 16;
  out->p = 1.0;
  out->sigma = 0.0;
  out->g_mode = 1;
  out->G1 = 1.0e4;
  out->E = 0;
  out->step_mode = 0;
  out->eta0 = 0.5;
  out->time = 1.0;
  out->scale_mode = 0;
  out->use_graph = 0;
  out->neigh_mode = 0;
  out->radius_scale = 1.0;
  return SCGR_OK;
}

scgr_status scgr_create(const scgr_params* params, void* cuda_stream, scgr_ctx** out) {
  if (!out) { g_create_error = "out is NULL"; return SCGR_ERR_INVALID_ARG; }
  *out = nullptr;
  std::string why;
  scgr_status st = check_params(params, why);
  if (st != SCGR_OK) { g_create_error = why; return st; }
  scgr_ctx* c = new (std::nothrow) scgr_ctx();
  if (!c) { g_create_error = "host allocation failed"; return SCGR_ERR_OOM; }
  c->prm = *params;
  c->stream = (cudaStream_t)cuda_stream;
  cudaError_t e = cudaGetDevice(&c->device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device);
  if (e == cudaSuccess) e = cudaMalloc((void**)&c->pose, sizeof(DevPose));
  if (e == cudaSuccess) e = cudaMalloc((void**)&c->stats, sizeof(DevStats));
  if (e == cudaSuccess) e = cudaMalloc((void**)&c->pose_eval, sizeof(DevPose));
  if (e == cudaSuccess) e = cudaMalloc((void**)&c->aux, sizeof(double) * 64);
  if (e == cudaSuccess) e = cudaMalloc((void**)&c->errword, sizeof(int));
  if (e == cudaSuccess) e = cudaMalloc((void**)&c->red, sizeof(double) * (RED_MAX_BLOCKS * 6 + 32));
  if (e == cudaSuccess) e = cudaMemsetAsync(c->errword, 0, sizeof(int), c->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->pose, 0, sizeof(DevPose), c->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->stats, 0, sizeof(DevStats), c->stream);
  if (e != cudaSuccess) {
    g_create_error = std::string("scgr_create: ") + cudaGetErrorString(e);
    cudaGetLastError();
    scgr_destroy(c);
    return e == cudaErrorMemoryAllocation ? SCGR_ERR_OOM : SCGR_ERR_CUDA;
  }
  c->qexp = (float)((params->p - 1.0) * 0.5);
  g_create_error.clear();
  *out = c;
  return SCGR_OK;
}

void scgr_destroy(scgr_ctx* c) {
  if (!c) return;
  if (c->stream) cudaStreamSynchronize(c->stream);
  else cudaDeviceSynchronize();
  drop_graph(c);
  for (cudaEvent_t e : c->ev) cudaEventDestroy(e);
  if (c->cap_stream) {
    cudaStreamSynchronize(c->cap_stream);
    cudaStreamDestroy(c->cap_stream);
  }
  if (c->join_in) cudaEventDestroy(c->join_in);
  if (c->join_out) cudaEventDestroy(c->join_out);
  if (c->bgexec) cudaGraphExecDestroy(c->bgexec);
  if (c->bgraph) cudaGraphDestroy(c->bgraph);
  DevBuf* bufs[] = {&c->X4, &c->Y4, &c->stage, &c->knnX, &c->knnY, &c->aX64, &c->aY64, &c->aX32,
                    &c->aY32, &c->Xr, &c->XA, &c->Y0r, &c->partial, &c->blockpart, &c->moved_stage,
                    &c->bX4, &c->bY4, &c->bknnX, &c->bknnY, &c->baX64, &c->baY64, &c->baX32, &c->baY32,
                    &c->bXr, &c->bXA, &c->bY0r, &c->bpartial, &c->bblockpart, &c->bpairs, &c->bitems,
                    &c->bcpair, &c->btabX, &c->btabY, &c->bxoff, &c->byoff, &c->bstats, &c->bposes,
                    &c->gcell, &c->gcount, &c->gstart, &c->gcursor, &c->gblock, &c->gsorted, &c->gsidx, &c->gbb,
                    &c->cd_key, &c->cd_moved, &c->wstore, &c->wupart, &c->wpartial, &c->mpart, &c->mom};
  for (DevBuf* b : bufs) release(*b);
  if (c->pose) cudaFree(c->pose);
  if (c->pose_eval) cudaFree(c->pose_eval);
  if (c->aux) cudaFree(c->aux);
  if (c->stats) cudaFree(c->stats);
  if (c->errword) cudaFree(c->errword);
  if (c->red) cudaFree(c->red);
  delete c;
}

const char* scgr_last_error(const scgr_ctx* c) {
  if (!c) return g_create_error.c_str();
  return c->err.c_str();
}

scgr_status scgr_set_reference(scgr_ctx* c, const float* xyz_dev, int64_t n) {
  return set_cloud(c, xyz_dev, n, false, true);
}
scgr_status scgr_set_reference_host(scgr_ctx* c, const float* xyz_host, int64_t n) {
  return set_cloud(c, xyz_host, n, true, true);
}
scgr_status scgr_set_template(scgr_ctx* c, const float* xyz_dev, int64_t m) {
  return set_cloud(c, xyz_dev, m, false, false);
}
scgr_status scgr_set_template_host(scgr_ctx* c, const float* xyz_host, int64_t m) {
  return set_cloud(c, xyz_host, m, true, false);
}

scgr_status scgr_compute_descriptors(scgr_ctx* c) {
  if (!c) return SCGR_ERR_INVALID_ARG;
  c->err.clear();
  if (!c->have_X || !c->have_Y) return fail(c, SCGR_ERR_STATE, "set the reference and the template first");
  const int k = c->prm.k;
  const int n = (int)c->n, m = (int)c->m;
  drop_graph(c);
  SCGR_CK(c, ensure(c->knnX, (size_t)n * k * sizeof(int32_t)));
  SCGR_CK(c, ensure(c->knnY, (size_t)m * k * sizeof(int32_t)));
  SCGR_CK(c, ensure(c->aX64, (size_t)n * sizeof(double)));
  SCGR_CK(c, ensure(c->aY64, (size_t)m * sizeof(double)));
  SCGR_CK(c, ensure(c->aX32, (size_t)n * sizeof(float)));
  SCGR_CK(c, ensure(c->aY32, (size_t)m * sizeof(float)));
  Launch L = c->L();
  const float4* X4 = (const float4*)c->X4.p;
  const float4* Y4 = (const float4*)c->Y4.p;
  DevStats* st = c->stats;
  SCGR_CK(c, launch_cloud_stats(L, X4, n, c->red, st->xbar, st->CX, &st->eX));
  SCGR_CK(c, launch_cloud_stats(L, Y4, m, c->red, st->ybar0, st->S0, &st->eY0));
  scgr_status cs = curvatures(c, c->prm.k, c->prm.radius_scale, 1.0);
  if (cs != SCGR_OK) return cs;
  c->npad = (c->n + 255) / 256 * 256;
  const int64_t mloc = c->rows >= 0 ? c->rows : c->m;
  c->fp = plan_force(mloc, c->npad, c->prm.p, c->num_sms, c->ftune);
  c->mpad = force_mpad(mloc, c->fp);
  SCGR_CK(c, ensure(c->Xr, (size_t)c->npad * sizeof(float4)));
  SCGR_CK(c, ensure(c->XA, (size_t)c->npad * sizeof(float2)));
  SCGR_CK(c, ensure(c->Y0r, (size_t)c->mpad * sizeof(float4)));
  SCGR_CK(c, ensure(c->partial, (size_t)c->fp.splits * c->mpad * sizeof(float4)));
  SCGR_CK(c, ensure(c->blockpart, (size_t)combine_blocks(c->mpad) * 13 * sizeof(double)));
  SCGR_CK(c, launch_records(L, X4, (const double*)c->aX64.p, n, (int)c->npad, Y4 + c->row0,
                            (const double*)c->aY64.p + c->row0, (int)mloc, (int)c->mpad, c->prm.g_mode, st,
                            (float4*)c->Xr.p, (float2*)c->XA.p, (float4*)c->Y0r.p));
  c->E_host = c->prm.E > 0 ? c->prm.E : 0;
  SCGR_CK(c, launch_pose_init(L, c->pose, st, c->E_host));
  c->iterations = 0;
  c->have_desc = true;
  return SCGR_OK;
}

scgr_status scgr_run(scgr_ctx* c, int iters) {
  if (!c) return SCGR_ERR_INVALID_ARG;
  c->err.clear();
  if (iters < 0) return fail(c, SCGR_ERR_INVALID_ARG, "iterations < 0");
  if (!c->have_desc) return fail(c, SCGR_ERR_STATE, "compute descriptors first");
  if (c->rows >= 0) return fail(c, SCGR_ERR_STATE, "a row range is set: iterate with scgr_step_partials/scgr_step_apply");
  if (iters == 0) return SCGR_OK;
  if (c->E_host <= 0) {
    c->E_host = iters;
    SCGR_CK(c, cudaMemcpyAsync(&c->pose->E, &c->E_host, sizeof(int), cudaMemcpyHostToDevice, c->stream));
  }
  if (c->prm.use_graph) {
    if (!c->cap_stream) {
      SCGR_CK(c, cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking));
      SCGR_CK(c, cudaEventCreateWithFlags(&c->join_in, cudaEventDisableTiming));
      SCGR_CK(c, cudaEventCreateWithFlags(&c->join_out, cudaEventDisableTiming));
    }
    if (c->graph_iters != iters) {
      drop_graph(c);
      const int64_t before = c->launches;
      cudaStream_t user = c->stream;
      c->stream = c->cap_stream;  // the launchers enqueue on c->stream
      cudaError_t e = cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal);
      scgr_status st = SCGR_OK;
      cudaGraph_t g = nullptr;
      if (e == cudaSuccess) {
        c->capturing = true;
        st = enqueue_iterations(c, iters);
        c->capturing = false;
        e = cudaStreamEndCapture(c->cap_stream, &g);
      }
      c->stream = user;
      c->launches = before;  // counted at replay
      if (st != SCGR_OK) { if (g) cudaGraphDestroy(g); return st; }
      if (e != cudaSuccess) return cuda_fail(c, e, "graph capture");
      c->graph = g;
      SCGR_CK(c, cudaGraphInstantiate(&c->gexec, c->graph, 0));
      c->graph_iters = iters;
    }
    // order the replay after earlier work on the user stream, and later work after it
    SCGR_CK(c, cudaEventRecord(c->join_in, c->stream));
    SCGR_CK(c, cudaStreamWaitEvent(c->cap_stream, c->join_in, 0));
    SCGR_CK(c, cudaGraphLaunch(c->gexec, c->cap_stream));
    SCGR_CK(c, cudaEventRecord(c->join_out, c->cap_stream));
    SCGR_CK(c, cudaStreamWaitEvent(c->stream, c->join_out, 0));
    const bool pf = c->fp.pmode == 1 && c->reuse_pose_free, mo = c->fp.pmode == 3 && c->reuse_pose_free;
    c->launches += pf ? 2 * (int64_t)iters + 1 : (mo ? 2 * (int64_t)iters + 2 : 3 * (int64_t)iters);
  } else {
    scgr_status st = enqueue_iterations(c, iters);
    if (st != SCGR_OK) return st;
  }
  c->iterations += iters;
  return SCGR_OK;
}

scgr_status scgr_sync(scgr_ctx* c) {
  if (!c) return SCGR_ERR_INVALID_ARG;
  c->err.clear();
  SCGR_CK(c, cudaStreamSynchronize(c->stream));
  return read_error_word(c);
}

scgr_status scgr_get_result(scgr_ctx* c, scgr_result* out) {
  if (!c || !out) return fail(c, SCGR_ERR_INVALID_ARG, "NULL argument");
  c->err.clear();
  if (!c->have_desc) return fail(c, SCGR_ERR_STATE, "compute descriptors first");
  DevPose h;
  SCGR_CK(c, cudaMemcpyAsync(&h, c->pose, sizeof(DevPose), cudaMemcpyDeviceToHost, c->stream));
  SCGR_CK(c, cudaStreamSynchronize(c->stream));
  std::memcpy(out->R, h.R, sizeof(out->R));
  std::memcpy(out->t, h.t, sizeof(out->t));
  out->s = h.s;
  out->iterations = h.it;
  out->degenerate_steps = h.degenerate;
  return read_error_word(c);
}

scgr_status scgr_get_moved(scgr_ctx* c, float* out) {
  if (!c || !out) return fail(c, SCGR_ERR_INVALID_ARG, "NULL argument");
  c->err.clear();
  if (!c->have_desc) return fail(c, SCGR_ERR_STATE, "compute descriptors first");
  SCGR_CK(c, launch_apply(c->L(), (const float4*)c->Y4.p, (int)c->m, c->pose, out));
  return SCGR_OK;
}

scgr_status scgr_get_moved_host(scgr_ctx* c, float* out) {
  if (!c || !out) return fail(c, SCGR_ERR_INVALID_ARG, "NULL argument");
  c->err.clear();
  if (!c->have_desc) return fail(c, SCGR_ERR_STATE, "compute descriptors first");
  SCGR_CK(c, ensure(c->moved_stage, (size_t)c->m * 3 * sizeof(float)));
  SCGR_CK(c, launch_apply(c->L(), (const float4*)c->Y4.p, (int)c->m, c->pose, (float*)c->moved_stage.p));
  SCGR_CK(c, cudaMemcpyAsync(out, c->moved_stage.p, (size_t)c->m * 3 * sizeof(float), cudaMemcpyDeviceToHost, c->stream));
  SCGR_CK(c, cudaStreamSynchronize(c->stream));
  return read_error_word(c);
}

scgr_status scgr_get_descriptors(scgr_ctx* c, int which, int32_t* knn_dev, float* a_dev) {
  if (!c) return SCGR_ERR_INVALID_ARG;
  c->err.clear();
  if (which != 0 && which != 1) return fail(c, SCGR_ERR_INVALID_ARG, "which must be 0 (reference) or 1 (template)");
  if (!c->have_desc) return fail(c, SCGR_ERR_STATE, "compute descriptors first");
  const int64_t n = which == 0 ? c->n : c->m;
  if (knn_dev && c->prm.neigh_mode != 0) return fail(c, SCGR_ERR_STATE, "no neighbour lists in the radius mode");
  if (knn_dev)
    SCGR_CK(c, cudaMemcpyAsync(knn_dev, which == 0 ? c->knnX.p : c->knnY.p, (size_t)n * c->prm.k * sizeof(int32_t),
                               cudaMemcpyDeviceToDevice, c->stream));
  if (a_dev)
    SCGR_CK(c, cudaMemcpyAsync(a_dev, which == 0 ? c->aX32.p : c->aY32.p, (size_t)n * sizeof(float),
                               cudaMemcpyDeviceToDevice, c->stream));
  return SCGR_OK;
}

scgr_status scgr_get_curvature64(scgr_ctx* c, int which, double* a64_dev) {
  if (!c || !a64_dev) return fail(c, SCGR_ERR_INVALID_ARG, "NULL argument");
  c->err.clear();
  if (which != 0 && which != 1) return fail(c, SCGR_ERR_INVALID_ARG, "which must be 0 or 1");
  if (!c->have_desc) return fail(c, SCGR_ERR_STATE, "compute descriptors first");
  const int64_t n = which == 0 ? c->n : c->m;
  SCGR_CK(c, cudaMemcpyAsync(a64_dev, which == 0 ? c->aX64.p : c->aY64.p, (size_t)n * sizeof(double),
                             cudaMemcpyDeviceToDevice, c->stream));
  return SCGR_OK;
}

scgr_status scgr_get_sigma(scgr_ctx* c, double* sigma_out) {
  if (!c || !sigma_out) return fail(c, SCGR_ERR_INVALID_ARG, "NULL argument");
  c->err.clear();
  if (!c->have_desc) return fail(c, SCGR_ERR_STATE, "compute descriptors first");
  SCGR_CK(c, cudaMemcpyAsync(sigma_out, &c->stats->sigma, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  SCGR_CK(c, cudaStreamSynchronize(c->stream));
  return read_error_word(c);
}

scgr_status scgr_forces(scgr_ctx* c, float* f4_dev) {
  if (!c || !f4_dev) return fail(c, SCGR_ERR_INVALID_ARG, "NULL argument");
  c->err.clear();
  if (!c->have_desc) return fail(c, SCGR_ERR_STATE, "compute descriptors first");
  scgr_status fs = force_launch(c);
  if (fs != SCGR_OK) return fs;
  const int mloc = (int)(c->rows >= 0 ? c->rows : c->m);
  SCGR_CK(c, launch_combine(c->L(), (const float4*)c->partial.p, c->fp.splits, (int)c->mpad, mloc,
                            (const float4*)c->Y0r.p, (const double*)c->aY64.p + c->row0, c->prm.g_mode, c->pose,
                            (float4*)f4_dev, (double*)c->blockpart.p));
  return SCGR_OK;
}

scgr_status scgr_potential_stored(scgr_ctx* c, const double pose7[7], double* U_out, double* grad_pose7,
                                  float* grad_xyz_dev) {
  if (!c || !pose7 || !U_out) return fail(c, SCGR_ERR_INVALID_ARG, "NULL argument");
  c->err.clear();
  if (!c->have_desc) return fail(c, SCGR_ERR_STATE, "compute descriptors first");
  if (c->rows >= 0) return fail(c, SCGR_ERR_STATE, "the potential needs the whole template (a row range is set)");
  for (int q = 0; q < 7; ++q)
    if (!std::isfinite(pose7[q])) return fail(c, SCGR_ERR_INVALID_ARG, "non-finite pose");
  if (!(pose7[6] > 0.0)) return fail(c, SCGR_ERR_INVALID_ARG, "scale must be > 0");
  const int n = (int)c->n, m = (int)c->m;
  const int nb = (n + 255) / 256;
  SCGR_CK(c, ensure(c->wstore, (size_t)n * m * sizeof(float)));
  SCGR_CK(c, ensure(c->wupart, (size_t)nb * ((m + 63) / 64) * sizeof(double)));
  SCGR_CK(c, ensure(c->wpartial, (size_t)c->mpad * sizeof(float4)));
  Launch L = c->L();
  double* d7 = c->aux + 48;
  SCGR_CK(c, cudaMemcpyAsync(d7, pose7, 7 * sizeof(double), cudaMemcpyHostToDevice, c->stream));
  SCGR_CK(c, launch_pose_from7(L, d7, c->pose_eval, c->stats));
  // forward: store w_ij and sum U
  SCGR_CK(c, launch_store_pairs(L, (const float2*)c->XA.p, (const float4*)c->Xr.p, n, (const float4*)c->Y0r.p,
                                (const double*)c->aY64.p, c->prm.g_mode, m, c->pose_eval, c->qexp,
                                (float*)c->wstore.p, (double*)c->wupart.p, c->aux + 3));
  if (grad_pose7 || grad_xyz_dev) {
    // backward from the stored terms
    SCGR_CK(c, launch_stored_rows(L, (const float*)c->wstore.p, n, m, (const float4*)c->Xr.p,
                                  (float4*)c->wpartial.p));
    SCGR_CK(c, launch_adjoint_combine(L, (const float4*)c->wpartial.p, 1, (int)c->mpad, m, (const float4*)c->Y0r.p,
                                      (const double*)c->aY64.p, c->prm.g_mode, c->pose_eval, grad_xyz_dev,
                                      (double*)c->blockpart.p));
    SCGR_CK(c, launch_column_sum13(L, (const double*)c->blockpart.p, combine_blocks(c->mpad), c->aux + 16));
    SCGR_CK(c, launch_adjoint_finish(L, c->aux + 16, d7, c->pose_eval, c->aux + 32));
  }
  double h[40];
  SCGR_CK(c, cudaMemcpyAsync(h, c->aux, 40 * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  SCGR_CK(c, cudaStreamSynchronize(c->stream));
  *U_out = h[3] / (c->prm.p + 1.0);
  if (grad_pose7)
    for (int q = 0; q < 7; ++q) grad_pose7[q] = h[32 + q];
  return read_error_word(c);
}

scgr_status scgr_force_vjp(scgr_ctx* c, const float* v_dev, float* grad_dev) {
  if (!c || !v_dev || !grad_dev) return fail(c, SCGR_ERR_INVALID_ARG, "NULL argument");
  c->err.clear();
  if (!c->have_desc) return fail(c, SCGR_ERR_STATE, "compute descriptors first");
  if (c->rows >= 0) return fail(c, SCGR_ERR_STATE, "the VJP needs the whole template (a row range is set)");
  SCGR_CK(c, launch_force_vjp(c->L(), (const float4*)c->Xr.p, (const float2*)c->XA.p, (int)(c->npad / FORCE_TJ),
                              (const float4*)c->Y0r.p, (const double*)c->aY64.p, c->prm.g_mode, (int)c->m, c->pose,
                              c->prm.p, v_dev, grad_dev));
  return SCGR_OK;
}

scgr_status scgr_nearest(scgr_ctx* c, const float* q_dev, int64_t nq, int32_t* idx_dev, float* key_dev) {
  if (!c || !q_dev || (!idx_dev && !key_dev)) return fail(c, SCGR_ERR_INVALID_ARG, "NULL argument");
  c->err.clear();
  if (!c->have_X) return fail(c, SCGR_ERR_STATE, "set the reference first");
  if (nq < 0 || nq > (int64_t(1) << 30)) return fail(c, SCGR_ERR_INVALID_ARG, "bad query count");
  SCGR_CK(c, launch_nearest(c->L(), (const float4*)c->X4.p, (int)c->n, q_dev, (int)nq, idx_dev, key_dev));
  return SCGR_OK;
}

scgr_status scgr_change_mask(scgr_ctx* c, double threshold, uint8_t* mask_dev, float* dist_dev) {
  if (!c || !mask_dev) return fail(c, SCGR_ERR_INVALID_ARG, "NULL argument");
  c->err.clear();
  if (!c->have_desc) return fail(c, SCGR_ERR_STATE, "compute descriptors first");
  if (!(threshold >= 0.0) || !std::isfinite(threshold)) return fail(c, SCGR_ERR_INVALID_ARG, "threshold must be >= 0");
  const int m = (int)c->m;
  SCGR_CK(c, ensure(c->cd_moved, (size_t)m * 3 * sizeof(float)));
  SCGR_CK(c, ensure(c->cd_key, (size_t)m * sizeof(float)));
  SCGR_CK(c, launch_apply(c->L(), (const float4*)c->Y4.p, m, c->pose, (float*)c->cd_moved.p));
  SCGR_CK(c, launch_nearest(c->L(), (const float4*)c->X4.p, (int)c->n, (const float*)c->cd_moved.p, m, nullptr,
                            (float*)c->cd_key.p));
  SCGR_CK(c, launch_threshold(c->L(), (const float*)c->cd_key.p, m, (float)(threshold * threshold), mask_dev,
                              dist_dev));
  return SCGR_OK;
}

scgr_status scgr_set_neighbourhood(scgr_ctx* c, int k, double radius_scale, double sigma_scale) {
  if (!c) return SCGR_ERR_INVALID_ARG;
  c->err.clear();
  if (!c->have_desc) return fail(c, SCGR_ERR_STATE, "compute descriptors first");
  if (c->prm.neigh_mode == 0 && (k < 3 || k > 32 || k > c->n || k > c->m))
    return fail(c, SCGR_ERR_INVALID_ARG, "k must be in [3, 32] and at most the cloud sizes");
  if (!(radius_scale > 0.0) || !(sigma_scale > 0.0) || !std::isfinite(radius_scale) || !std::isfinite(sigma_scale))
    return fail(c, SCGR_ERR_INVALID_ARG, "scales must be finite and > 0");
  drop_graph(c);
  scgr_status cs = curvatures(c, c->prm.neigh_mode == 0 ? k : c->prm.k, radius_scale, sigma_scale);
  if (cs != SCGR_OK) return cs;
  const int64_t mloc = c->rows >= 0 ? c->rows : c->m;
  SCGR_CK(c, launch_records(c->L(), (const float4*)c->X4.p, (const double*)c->aX64.p, (int)c->n, (int)c->npad,
                            (const float4*)c->Y4.p + c->row0, (const double*)c->aY64.p + c->row0, (int)mloc,
                            (int)c->mpad, c->prm.g_mode, c->stats, (float4*)c->Xr.p, (float2*)c->XA.p,
                            (float4*)c->Y0r.p));
  return SCGR_OK;
}

scgr_status scgr_set_curvature(scgr_ctx* c, int which, const double* a64_dev) {
  if (!c || !a64_dev) return fail(c, SCGR_ERR_INVALID_ARG, "NULL argument");
  c->err.clear();
  if (which != 0 && which != 1) return fail(c, SCGR_ERR_INVALID_ARG, "which must be 0 or 1");
  if (!c->have_desc) return fail(c, SCGR_ERR_STATE, "compute descriptors first");
  const int n = (int)(which == 0 ? c->n : c->m);
  DevBuf& a64 = which == 0 ? c->aX64 : c->aY64;
  DevBuf& a32 = which == 0 ? c->aX32 : c->aY32;
  drop_graph(c);
  Launch L = c->L();
  SCGR_CK(c, cudaMemcpyAsync(a64.p, a64_dev, (size_t)n * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
  SCGR_CK(c, launch_check_curvature(L, (const double*)a64.p, n, (float*)a32.p, c->errword));
  DevStats* st = c->stats;
  SCGR_CK(c, launch_sigma(L, (const double*)c->aX64.p, (int)c->n, c->prm.sigma, c->red, &st->sigma, &st->asum[0]));
  SCGR_CK(c, launch_records(L, (const float4*)c->X4.p, (const double*)c->aX64.p, (int)c->n, (int)c->npad,
                            (const float4*)c->Y4.p, (const double*)c->aY64.p, (int)c->m, (int)c->mpad,
                            c->prm.g_mode, st, (float4*)c->Xr.p, (float2*)c->XA.p, (float4*)c->Y0r.p));
  c->E_host = c->prm.E > 0 ? c->prm.E : 0;
  SCGR_CK(c, launch_pose_init(L, c->pose, st, c->E_host));
  c->iterations = 0;
  return SCGR_OK;
}

scgr_status scgr_set_force_timing(scgr_ctx* c, int enable) {
  if (!c) return SCGR_ERR_INVALID_ARG;
  c->err.clear();
  SCGR_CK(c, cudaStreamSynchronize(c->stream));
  c->ev_used = 0;
  c->timed_ms = 0.0;
  c->timed_launches = 0;
  c->timing = enable != 0;
  return SCGR_OK;
}

scgr_status scgr_get_force_timing(scgr_ctx* c, int64_t* launches, double* total_ms) {
  if (!c || !launches || !total_ms) return fail(c, SCGR_ERR_INVALID_ARG, "NULL argument");
  c->err.clear();
  SCGR_CK(c, cudaStreamSynchronize(c->stream));
  scgr_status st = collect_timing(c);
  if (st != SCGR_OK) return st;
  *launches = c->timed_launches;
  *total_ms = c->timed_ms;
  return SCGR_OK;
}

scgr_status scgr_get_state(scgr_ctx* c, scgr_state* out) {
  if (!c || !out) return fail(c, SCGR_ERR_INVALID_ARG, "NULL argument");
  c->err.clear();
  if (!c->have_desc) return fail(c, SCGR_ERR_STATE, "compute descriptors first");
  DevPose h;
  double sigma = 0;
  SCGR_CK(c, cudaMemcpyAsync(&h, c->pose, sizeof(DevPose), cudaMemcpyDeviceToHost, c->stream));
  SCGR_CK(c, cudaMemcpyAsync(&sigma, &c->stats->sigma, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  SCGR_CK(c, cudaStreamSynchronize(c->stream));
  std::memcpy(out->R, h.R, sizeof(out->R));
  std::memcpy(out->t, h.t, sizeof(out->t));
  out->s = h.s;
  out->iteration = h.it;
  out->E = h.E;
  out->degenerate_steps = h.degenerate;
  out->sigma = sigma;
  return read_error_word(c);
}

scgr_status scgr_set_state(scgr_ctx* c, const scgr_state* in) {
  if (!c || !in) return fail(c, SCGR_ERR_INVALID_ARG, "NULL argument");
  c->err.clear();
  if (!c->have_desc) return fail(c, SCGR_ERR_STATE, "compute descriptors first");
  for (int q = 0; q < 9; ++q)
    if (!std::isfinite(in->R[q])) return fail(c, SCGR_ERR_INVALID_ARG, "non-finite R");
  for (int q = 0; q < 3; ++q)
    if (!std::isfinite(in->t[q])) return fail(c, SCGR_ERR_INVALID_ARG, "non-finite t");
  if (!(in->s > 0.0) || !std::isfinite(in->s)) return fail(c, SCGR_ERR_INVALID_ARG, "s must be > 0");
  if (in->iteration < 0 || in->E < 0) return fail(c, SCGR_ERR_INVALID_ARG, "negative iteration or E");
  DevPose h;
  SCGR_CK(c, cudaMemcpyAsync(&h, c->pose, sizeof(DevPose), cudaMemcpyDeviceToHost, c->stream));
  SCGR_CK(c, cudaStreamSynchronize(c->stream));
  std::memcpy(h.R, in->R, sizeof(h.R));
  std::memcpy(h.t, in->t, sizeof(h.t));
  h.s = in->s;
  h.it = in->iteration;
  h.E = in->E;
  h.degenerate = in->degenerate_steps;
  c->E_host = in->E;
  SCGR_CK(c, cudaMemcpyAsync(c->pose, &h, sizeof(DevPose), cudaMemcpyHostToDevice, c->stream));
  SCGR_CK(c, launch_pose_refresh(c->L(), c->pose, c->stats));
  SCGR_CK(c, cudaStreamSynchronize(c->stream));
  drop_graph(c);
  return SCGR_OK;
}

scgr_status scgr_potential(scgr_ctx* c, const double pose7[7], double* U_out, double* grad_pose7,
                           float* grad_xyz_dev) {
  if (!c || !pose7 || !U_out) return fail(c, SCGR_ERR_INVALID_ARG, "NULL argument");
  c->err.clear();
  if (!c->have_desc) return fail(c, SCGR_ERR_STATE, "compute descriptors first");
  for (int q = 0; q < 7; ++q)
    if (!std::isfinite(pose7[q])) return fail(c, SCGR_ERR_INVALID_ARG, "non-finite pose");
  if (!(pose7[6] > 0.0)) return fail(c, SCGR_ERR_INVALID_ARG, "scale must be > 0");
  if (c->rows >= 0) return fail(c, SCGR_ERR_STATE, "the potential needs the whole template (a row range is set)");
  Launch L = c->L();
  double* d7 = c->aux + 48;
  SCGR_CK(c, cudaMemcpyAsync(d7, pose7, 7 * sizeof(double), cudaMemcpyHostToDevice, c->stream));
  SCGR_CK(c, launch_pose_from7(L, d7, c->pose_eval, c->stats));
  const int ntiles = (int)(c->npad / c->fp.tile_j);
  const int nb = combine_blocks(c->mpad);
  // forward: the force kernel with the distance exponent p + 1 accumulates
  // sum_j g d^(p+1); U = sum_i aY_i (that sum) / (p + 1)
  ForcePlan fu = c->fp;
  const double eU = c->prm.p + 1.0;
  fu.pmode = (eU == 2.0) ? 3 : 0;
  SCGR_CK(c, launch_force(L, fu, (const float4*)c->Xr.p, (const float2*)c->XA.p, ntiles, (const float4*)c->Y0r.p,
                          (int)c->mpad, c->pose_eval, (float)(0.5 * eU), (float4*)c->partial.p));
  SCGR_CK(c, launch_combine(L, (const float4*)c->partial.p, fu.splits, (int)c->mpad, (int)c->m,
                            (const float4*)c->Y0r.p, (const double*)c->aY64.p, c->prm.g_mode, c->pose_eval,
                            nullptr, (double*)c->blockpart.p));
  SCGR_CK(c, launch_column_sum13(L, (const double*)c->blockpart.p, nb, c->aux));
  if (grad_pose7 || grad_xyz_dev) {
    // adjoint: recompute the pair tiles at the same pose for G_i = -f_i
    SCGR_CK(c, launch_force(L, c->fp, (const float4*)c->Xr.p, (const float2*)c->XA.p, ntiles,
                            (const float4*)c->Y0r.p, (int)c->mpad, c->pose_eval, c->qexp, (float4*)c->partial.p));
    SCGR_CK(c, launch_adjoint_combine(L, (const float4*)c->partial.p, c->fp.splits, (int)c->mpad, (int)c->m,
                                      (const float4*)c->Y0r.p, (const double*)c->aY64.p, c->prm.g_mode,
                                      c->pose_eval, grad_xyz_dev, (double*)c->blockpart.p));
    SCGR_CK(c, launch_column_sum13(L, (const double*)c->blockpart.p, nb, c->aux + 16));
    SCGR_CK(c, launch_adjoint_finish(L, c->aux + 16, d7, c->pose_eval, c->aux + 32));
  }
  double h[40];
  SCGR_CK(c, cudaMemcpyAsync(h, c->aux, 40 * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  SCGR_CK(c, cudaStreamSynchronize(c->stream));
  *U_out = h[3] / eU;
  if (grad_pose7)
    for (int q = 0; q < 7; ++q) grad_pose7[q] = h[32 + q];
  return read_error_word(c);
}

scgr_status scgr_set_row_range(scgr_ctx* c, int64_t row0, int64_t rows) {
  if (!c) return SCGR_ERR_INVALID_ARG;
  c->err.clear();
  if (!c->have_Y) return fail(c, SCGR_ERR_STATE, "set the template first");
  if (row0 < 0 || rows < 1 || row0 + rows > c->m) return fail(c, SCGR_ERR_INVALID_ARG, "row range outside the template");
  c->row0 = row0;
  c->rows = rows;
  c->have_desc = false;
  return SCGR_OK;
}

scgr_status scgr_step_partials(scgr_ctx* c, double out13[13]) {
  if (!c || !out13) return fail(c, SCGR_ERR_INVALID_ARG, "NULL argument");
  c->err.clear();
  if (!c->have_desc) return fail(c, SCGR_ERR_STATE, "compute descriptors first");
  if (c->E_host <= 0) return fail(c, SCGR_ERR_STATE, "set params.E for stepwise iteration");
  const int mloc = (int)(c->rows >= 0 ? c->rows : c->m);
  scgr_status fs = force_launch(c);
  if (fs != SCGR_OK) return fs;
  SCGR_CK(c, launch_combine(c->L(), (const float4*)c->partial.p, c->fp.splits, (int)c->mpad, mloc,
                            (const float4*)c->Y0r.p, (const double*)c->aY64.p + c->row0, c->prm.g_mode, c->pose,
                            nullptr, (double*)c->blockpart.p));
  SCGR_CK(c, launch_column_sum13(c->L(), (const double*)c->blockpart.p, combine_blocks(c->mpad), c->aux));
  SCGR_CK(c, cudaMemcpyAsync(out13, c->aux, 13 * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  SCGR_CK(c, cudaStreamSynchronize(c->stream));
  return read_error_word(c);
}

scgr_status scgr_step_apply(scgr_ctx* c, const double tot13[13]) {
  if (!c || !tot13) return fail(c, SCGR_ERR_INVALID_ARG, "NULL argument");
  c->err.clear();
  if (!c->have_desc) return fail(c, SCGR_ERR_STATE, "compute descriptors first");
  if (c->E_host <= 0) return fail(c, SCGR_ERR_STATE, "set params.E for stepwise iteration");
  for (int q = 0; q < 13; ++q)
    if (!std::isfinite(tot13[q])) return fail(c, SCGR_ERR_INVALID_ARG, "non-finite totals");
  SCGR_CK(c, cudaMemcpyAsync(c->aux + 16, tot13, 13 * sizeof(double), cudaMemcpyHostToDevice, c->stream));
  SCGR_CK(c, launch_finalize(c->L(), c->aux + 16, 1, c->pose, c->stats, step_params(c), c->errword));
  SCGR_CK(c, cudaStreamSynchronize(c->stream));
  c->iterations += 1;
  return read_error_word(c);
}

scgr_status scgr_get_plan(scgr_ctx* c, int out[5]) {
  if (!c || !out) return fail(c, SCGR_ERR_INVALID_ARG, "NULL argument");
  c->err.clear();
  if (!c->have_desc) return fail(c, SCGR_ERR_STATE, "compute descriptors first");
  out[0] = c->fp.P;
  out[1] = c->fp.tpb;
  out[2] = c->fp.splits;
  out[3] = c->fp.iblocks;
  out[4] = c->fp.occ;
  return SCGR_OK;
}

scgr_status scgr_set_tuning(scgr_ctx* c, int key, int value) {
  if (!c) return SCGR_ERR_INVALID_ARG;
  c->err.clear();
  if (key == SCGR_TUNE_FORCE_P) {
    if (value != 0 && value != 1 && value != 2 && value != 4) return fail(c, SCGR_ERR_INVALID_ARG, "P must be 0, 1, 2 or 4");
    c->ftune.P = value;
    return c->have_desc ? replan(c) : SCGR_OK;
  }
  if (key == SCGR_TUNE_FORCE_TPB) {
    if (value != 0 && value != 128 && value != 256) return fail(c, SCGR_ERR_INVALID_ARG, "threads per block must be 0, 128 or 256");
    c->ftune.tpb = value;
    return c->have_desc ? replan(c) : SCGR_OK;
  }
  if (key == SCGR_TUNE_FORCE_OCC) {
    if (value != 0 && value != 1) return fail(c, SCGR_ERR_INVALID_ARG, "occupancy variant must be 0 or 1");
    c->ftune.occ = value;
    return c->have_desc ? replan(c) : SCGR_OK;
  }
  if (key == SCGR_TUNE_FORCE_SPLITS) {
    if (value < 0 || value > 4096) return fail(c, SCGR_ERR_INVALID_ARG, "splits must be in [0, 4096]");
    c->ftune.splits = value;
    return c->have_desc ? replan(c) : SCGR_OK;
  }
  if (key == SCGR_TUNE_REUSE_POSE_FREE) {
    if (value != 0 && value != 1) return fail(c, SCGR_ERR_INVALID_ARG, "value must be 0 or 1");
    c->reuse_pose_free = value;
    drop_graph(c);
    return SCGR_OK;
  }
  if (key == SCGR_TUNE_KNN_GRID_MIN) {
    if (value < 0) return fail(c, SCGR_ERR_INVALID_ARG, "grid threshold must be >= 0");
    c->knn_grid_min = value;
    return SCGR_OK;
  }
  if (key == SCGR_TUNE_BATCH_P) {
    if (value != 1 && value != 2) return fail(c, SCGR_ERR_INVALID_ARG, "batch points per thread must be 1 or 2");
    c->batch_P = value;
    return SCGR_OK;
  }
  if (key == SCGR_TUNE_BATCH_CHUNK_TILES) {
    if (value < 1 || value > 4096) return fail(c, SCGR_ERR_INVALID_ARG, "chunk tiles must be in [1, 4096]");
    c->batch_chunk_tiles = value;
    return SCGR_OK;
  }
  return fail(c, SCGR_ERR_INVALID_ARG, "unknown tuning key");
}

scgr_status scgr_batch_run(scgr_ctx* c, int npairs, const int64_t* ref_off, const float* ref_xyz_dev,
                           const int64_t* tmp_off, const float* tmp_xyz_dev, int iterations,
                           scgr_result* results) {
  if (!c) return SCGR_ERR_INVALID_ARG;
  c->err.clear();
  if (npairs < 1 || !ref_off || !tmp_off || !ref_xyz_dev || !tmp_xyz_dev || !results)
    return fail(c, SCGR_ERR_INVALID_ARG, "NULL argument or npairs < 1");
  if (iterations < 0) return fail(c, SCGR_ERR_INVALID_ARG, "iterations < 0");
  const int k = c->prm.k;
  if (ref_off[0] != 0 || tmp_off[0] != 0) return fail(c, SCGR_ERR_INVALID_ARG, "offsets must start at 0");
  for (int p = 0; p < npairs; ++p) {
    if (ref_off[p + 1] - ref_off[p] < k) return fail(c, SCGR_ERR_INVALID_ARG, "a reference has fewer than k points");
    if (tmp_off[p + 1] - tmp_off[p] < std::max(k, 3)) return fail(c, SCGR_ERR_INVALID_ARG, "a template has fewer than max(k, 3) points");
  }
  const int64_t Ntot = ref_off[npairs], Mtot = tmp_off[npairs];
  if (Ntot >= (int64_t(1) << 30) || Mtot >= (int64_t(1) << 30)) return fail(c, SCGR_ERR_INVALID_ARG, "too many points");

  // ---- host plan: per-pair geometry, work items (longest first), tables
  const int CT = c->batch_chunk_tiles;
  const int FB = 128 * c->batch_P;  // template points per batched force block
  std::vector<BatchPair> pairs(npairs);
  std::vector<int4> items;
  std::vector<int> cpair;
  std::vector<int2> tabX, tabY;
  int64_t xt = 0, yb = 0, pb = 0;
  int cb = 0;
  for (int p = 0; p < npairs; ++p) {
    BatchPair& bp = pairs[p];
    bp.x0 = ref_off[p];
    bp.n = ref_off[p + 1] - ref_off[p];
    bp.y0 = tmp_off[p];
    bp.m = tmp_off[p + 1] - tmp_off[p];
    bp.ntiles = (int)((bp.n + FORCE_TJ - 1) / FORCE_TJ);
    bp.xtile0 = xt;
    xt += bp.ntiles;
    bp.mpad = (bp.m + 255) / 256 * 256;
    bp.ybase = yb;
    yb += bp.mpad;
    bp.chunks = (bp.ntiles + CT - 1) / CT;
    bp.pbase = pb;
    pb += (int64_t)bp.chunks * bp.mpad;
    bp.cblk0 = cb;
    bp.ncblk = (int)(bp.mpad / 256);
    cb += bp.ncblk;
    for (int q = 0; q < bp.ncblk; ++q) cpair.push_back(p);
    const int fblocks = (int)((bp.m + FB - 1) / FB);
    for (int b = 0; b < fblocks; ++b)
      for (int ch = 0; ch < bp.chunks; ++ch) {
        const int tiles = std::min(CT, bp.ntiles - ch * CT);
        const int pts = (int)std::min<int64_t>(FB, bp.m - (int64_t)b * FB);
        items.push_back(make_int4(p, b, ch, tiles * pts));
      }
    for (int64_t q0 = 0; q0 < bp.n; q0 += 128) tabX.push_back(make_int2(p, (int)q0));
    for (int64_t q0 = 0; q0 < bp.m; q0 += 128) tabY.push_back(make_int2(p, (int)q0));
  }
  std::stable_sort(items.begin(), items.end(), [](const int4& a, const int4& b) { return a.w > b.w; });
  std::vector<int64_t> xoff(ref_off, ref_off + npairs + 1), yoff(tmp_off, tmp_off + npairs + 1);

  // ---- device buffers
  SCGR_CK(c, ensure(c->bX4, (size_t)Ntot * sizeof(float4)));
  SCGR_CK(c, ensure(c->bY4, (size_t)Mtot * sizeof(float4)));
  SCGR_CK(c, ensure(c->bknnX, (size_t)Ntot * k * sizeof(int32_t)));
  SCGR_CK(c, ensure(c->bknnY, (size_t)Mtot * k * sizeof(int32_t)));
  SCGR_CK(c, ensure(c->baX64, (size_t)Ntot * sizeof(double)));
  SCGR_CK(c, ensure(c->baY64, (size_t)Mtot * sizeof(double)));
  SCGR_CK(c, ensure(c->baX32, (size_t)Ntot * sizeof(float)));
  SCGR_CK(c, ensure(c->baY32, (size_t)Mtot * sizeof(float)));
  SCGR_CK(c, ensure(c->bXr, (size_t)xt * FORCE_TJ * sizeof(float4)));
  SCGR_CK(c, ensure(c->bXA, (size_t)xt * FORCE_TJ * sizeof(float2)));
  SCGR_CK(c, ensure(c->bY0r, (size_t)yb * sizeof(float4)));
  SCGR_CK(c, ensure(c->bpartial, (size_t)pb * sizeof(float4)));
  SCGR_CK(c, ensure(c->bblockpart, (size_t)cb * 13 * sizeof(double)));
  SCGR_CK(c, ensure(c->bpairs, pairs.size() * sizeof(BatchPair)));
  SCGR_CK(c, ensure(c->bitems, items.size() * sizeof(int4)));
  SCGR_CK(c, ensure(c->bcpair, cpair.size() * sizeof(int)));
  SCGR_CK(c, ensure(c->btabX, tabX.size() * sizeof(int2)));
  SCGR_CK(c, ensure(c->btabY, tabY.size() * sizeof(int2)));
  SCGR_CK(c, ensure(c->bxoff, xoff.size() * sizeof(int64_t)));
  SCGR_CK(c, ensure(c->byoff, yoff.size() * sizeof(int64_t)));
  SCGR_CK(c, ensure(c->bstats, (size_t)npairs * sizeof(DevStats)));
  SCGR_CK(c, ensure(c->bposes, (size_t)npairs * sizeof(DevPose)));
  cudaStream_t st = c->stream;
  SCGR_CK(c, cudaMemcpyAsync(c->bpairs.p, pairs.data(), pairs.size() * sizeof(BatchPair), cudaMemcpyHostToDevice, st));
  SCGR_CK(c, cudaMemcpyAsync(c->bitems.p, items.data(), items.size() * sizeof(int4), cudaMemcpyHostToDevice, st));
  SCGR_CK(c, cudaMemcpyAsync(c->bcpair.p, cpair.data(), cpair.size() * sizeof(int), cudaMemcpyHostToDevice, st));
  SCGR_CK(c, cudaMemcpyAsync(c->btabX.p, tabX.data(), tabX.size() * sizeof(int2), cudaMemcpyHostToDevice, st));
  SCGR_CK(c, cudaMemcpyAsync(c->btabY.p, tabY.data(), tabY.size() * sizeof(int2), cudaMemcpyHostToDevice, st));
  SCGR_CK(c, cudaMemcpyAsync(c->bxoff.p, xoff.data(), xoff.size() * sizeof(int64_t), cudaMemcpyHostToDevice, st));
  SCGR_CK(c, cudaMemcpyAsync(c->byoff.p, yoff.data(), yoff.size() * sizeof(int64_t), cudaMemcpyHostToDevice, st));

  // ---- descriptors for every cloud, in one launch per stage
  Launch L = c->L();
  const BatchPair* dpairs = (const BatchPair*)c->bpairs.p;
  SCGR_CK(c, launch_pack(L, ref_xyz_dev, Ntot, (float4*)c->bX4.p, c->errword));
  SCGR_CK(c, launch_pack(L, tmp_xyz_dev, Mtot, (float4*)c->bY4.p, c->errword));
  SCGR_CK(c, launch_knn_multi(L, (const float4*)c->bX4.p, (const int64_t*)c->bxoff.p, (const int2*)c->btabX.p,
                              (int)tabX.size(), k, (int32_t*)c->bknnX.p));
  SCGR_CK(c, launch_knn_multi(L, (const float4*)c->bY4.p, (const int64_t*)c->byoff.p, (const int2*)c->btabY.p,
                              (int)tabY.size(), k, (int32_t*)c->bknnY.p));
  SCGR_CK(c, launch_curvature(L, (const float4*)c->bX4.p, (const int32_t*)c->bknnX.p, (int)Ntot, k,
                              (double*)c->baX64.p, (float*)c->baX32.p));
  SCGR_CK(c, launch_curvature(L, (const float4*)c->bY4.p, (const int32_t*)c->bknnY.p, (int)Mtot, k,
                              (double*)c->baY64.p, (float*)c->baY32.p));
  SCGR_CK(c, launch_stats_multi(L, (const float4*)c->bX4.p, (const float4*)c->bY4.p, (const double*)c->baX64.p,
                                dpairs, npairs, c->prm.sigma, (DevStats*)c->bstats.p));
  SCGR_CK(c, launch_records_multi(L, (const float4*)c->bX4.p, (const double*)c->baX64.p, (const float4*)c->bY4.p,
                                  (const double*)c->baY64.p, dpairs, npairs, c->prm.g_mode,
                                  (const DevStats*)c->bstats.p, (float4*)c->bXr.p, (float2*)c->bXA.p,
                                  (float4*)c->bY0r.p));
  const int E = c->prm.E > 0 ? c->prm.E : std::max(iterations, 1);
  SCGR_CK(c, launch_pose_init_multi(L, (DevPose*)c->bposes.p, (const DevStats*)c->bstats.p, npairs, E));

  // ---- iterations: three launches per iteration for all pairs
  StepParams sp = step_params(c);
  const int pmode = (c->prm.p == 1.0) ? 1 : (c->prm.p == 2.0) ? 2 : (c->prm.p == 3.0) ? 3 : 0;
  auto enqueue = [&](Launch LL) -> scgr_status {
    for (int t = 0; t < iterations; ++t) {
      SCGR_CK(c, launch_force_batch(LL, pmode, c->batch_P, (int)items.size(), (const int4*)c->bitems.p, dpairs,
                                    (const float4*)c->bXr.p, (const float2*)c->bXA.p, (const float4*)c->bY0r.p,
                                    (const DevPose*)c->bposes.p, c->qexp, (float4*)c->bpartial.p, CT));
      SCGR_CK(c, launch_combine_batch(LL, cb, (const int*)c->bcpair.p, dpairs, (const float4*)c->bpartial.p,
                                      (const float4*)c->bY0r.p, (const double*)c->baY64.p, c->prm.g_mode,
                                      (const DevPose*)c->bposes.p, (double*)c->bblockpart.p));
      SCGR_CK(c, launch_finalize_multi(LL, (const double*)c->bblockpart.p, dpairs, npairs, (DevPose*)c->bposes.p,
                                       (const DevStats*)c->bstats.p, sp, c->errword));
    }
    return SCGR_OK;
  };
  if (iterations > 0) {
    if (c->prm.use_graph) {
      if (!c->cap_stream) {
        SCGR_CK(c, cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking));
        SCGR_CK(c, cudaEventCreateWithFlags(&c->join_in, cudaEventDisableTiming));
        SCGR_CK(c, cudaEventCreateWithFlags(&c->join_out, cudaEventDisableTiming));
      }
      if (c->bgexec) cudaGraphExecDestroy(c->bgexec);
      if (c->bgraph) cudaGraphDestroy(c->bgraph);
      c->bgexec = nullptr;
      c->bgraph = nullptr;
      SCGR_CK(c, cudaEventRecord(c->join_in, c->stream));
      SCGR_CK(c, cudaStreamWaitEvent(c->cap_stream, c->join_in, 0));
      const int64_t before = c->launches;
      cudaError_t e = cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal);
      scgr_status stq = SCGR_OK;
      cudaGraph_t g = nullptr;
      if (e == cudaSuccess) {
        stq = enqueue(Launch{c->cap_stream, &c->launches});
        e = cudaStreamEndCapture(c->cap_stream, &g);
      }
      c->launches = before;
      if (stq != SCGR_OK) { if (g) cudaGraphDestroy(g); return stq; }
      if (e != cudaSuccess) return cuda_fail(c, e, "batch graph capture");
      c->bgraph = g;
      SCGR_CK(c, cudaGraphInstantiate(&c->bgexec, c->bgraph, 0));
      SCGR_CK(c, cudaGraphLaunch(c->bgexec, c->cap_stream));
      SCGR_CK(c, cudaEventRecord(c->join_out, c->cap_stream));
      SCGR_CK(c, cudaStreamWaitEvent(c->stream, c->join_out, 0));
      c->launches += 3 * (int64_t)iterations;
    } else {
      scgr_status stq = enqueue(L);
      if (stq != SCGR_OK) return stq;
    }
  }

  // ---- results
  std::vector<DevPose> hp(npairs);
  SCGR_CK(c, cudaMemcpyAsync(hp.data(), c->bposes.p, (size_t)npairs * sizeof(DevPose), cudaMemcpyDeviceToHost, st));
  SCGR_CK(c, cudaStreamSynchronize(st));
  for (int p = 0; p < npairs; ++p) {
    std::memcpy(results[p].R, hp[p].R, sizeof(results[p].R));
    std::memcpy(results[p].t, hp[p].t, sizeof(results[p].t));
    results[p].s = hp[p].s;
    results[p].iterations = hp[p].it;
    results[p].degenerate_steps = hp[p].degenerate;
  }
  return read_error_word(c);
}

int64_t scgr_launch_count(const scgr_ctx* c) { return c ? c->launches : -1; }

}  // extern "C"
