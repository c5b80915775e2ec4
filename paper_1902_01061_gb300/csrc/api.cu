// C ABI of the scgr library: context, buffers, argument checks and the
// launch sequence of the method (see include/scgr.h for the contract).
#include <cuda_runtime.h>

#include <climits>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
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
  bool have_X = false, have_Y = false, have_desc = false;
  int E_host = 0;          // Eq. 12 horizon in use (0: not fixed yet)
  int iterations = 0;      // iterations enqueued since the descriptors
  int64_t launches = 0;
  ForcePlan fp{};
  float qexp = 0.f;        // (p - 1) / 2, exponent of d^2 in the weight

  DevBuf X4, Y4, stage, knnX, knnY, aX64, aY64, aX32, aY32, Xr, XA, Y0r, partial, blockpart,
      moved_stage;
  DevPose* pose = nullptr;
  DevStats* stats = nullptr;
  int* errword = nullptr;
  double* red = nullptr;   // reduction scratch

  cudaGraph_t graph = nullptr;
  cudaGraphExec_t gexec = nullptr;
  int graph_iters = -1;
  bool capturing = false;
  cudaStream_t cap_stream = nullptr;  // capture / replay stream (never the legacy stream)
  cudaEvent_t join_in = nullptr, join_out = nullptr;

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

scgr_status enqueue_iterations(scgr_ctx* c, int iters) {
  const int nb = combine_blocks(c->mpad);
  const StepParams sp = step_params(c);
  for (int t = 0; t < iters; ++t) {
    scgr_status fs = force_launch(c);
    if (fs != SCGR_OK) return fs;
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
  DevBuf* bufs[] = {&c->X4, &c->Y4, &c->stage, &c->knnX, &c->knnY, &c->aX64, &c->aY64, &c->aX32,
                    &c->aY32, &c->Xr, &c->XA, &c->Y0r, &c->partial, &c->blockpart, &c->moved_stage};
  for (DevBuf* b : bufs) release(*b);
  if (c->pose) cudaFree(c->pose);
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
  SCGR_CK(c, launch_knn(L, X4, n, k, (int32_t*)c->knnX.p));
  SCGR_CK(c, launch_knn(L, Y4, m, k, (int32_t*)c->knnY.p));
  SCGR_CK(c, launch_curvature(L, X4, (const int32_t*)c->knnX.p, n, k, (double*)c->aX64.p, (float*)c->aX32.p));
  SCGR_CK(c, launch_curvature(L, Y4, (const int32_t*)c->knnY.p, m, k, (double*)c->aY64.p, (float*)c->aY32.p));
  DevStats* st = c->stats;
  SCGR_CK(c, launch_cloud_stats(L, X4, n, c->red, st->xbar, st->CX, &st->eX));
  SCGR_CK(c, launch_cloud_stats(L, Y4, m, c->red, st->ybar0, st->S0, &st->eY0));
  SCGR_CK(c, launch_sigma(L, (const double*)c->aX64.p, n, c->prm.sigma, c->red, &st->sigma, &st->asum[0]));
  c->npad = (c->n + 255) / 256 * 256;
  c->fp = plan_force(c->m, c->npad, c->prm.p, c->num_sms);
  c->mpad = force_mpad(c->m, c->fp);
  SCGR_CK(c, ensure(c->Xr, (size_t)c->npad * sizeof(float4)));
  SCGR_CK(c, ensure(c->XA, (size_t)c->npad * sizeof(float2)));
  SCGR_CK(c, ensure(c->Y0r, (size_t)c->mpad * sizeof(float4)));
  SCGR_CK(c, ensure(c->partial, (size_t)c->fp.splits * c->mpad * sizeof(float4)));
  SCGR_CK(c, ensure(c->blockpart, (size_t)combine_blocks(c->mpad) * 13 * sizeof(double)));
  SCGR_CK(c, launch_records(L, X4, (const double*)c->aX64.p, n, (int)c->npad, Y4, (const double*)c->aY64.p, m,
                            (int)c->mpad, c->prm.g_mode, st, (float4*)c->Xr.p, (float2*)c->XA.p, (float4*)c->Y0r.p));
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
    c->launches += 3 * (int64_t)iters;
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
  SCGR_CK(c, launch_combine(c->L(), (const float4*)c->partial.p, c->fp.splits, (int)c->mpad, (int)c->m,
                            (const float4*)c->Y0r.p, (const double*)c->aY64.p, c->prm.g_mode, c->pose,
                            (float4*)f4_dev, (double*)c->blockpart.p));
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

int64_t scgr_launch_count(const scgr_ctx* c) { return c ? c->launches : -1; }

}  // extern "C"
