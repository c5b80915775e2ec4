// C ABI of the scgr library: context lifecycle, clouds, descriptors, the
// iteration loop, results, state and tuning (see include/scgr.h for the
// contract).  The differentiation, batching and extra entry points live in
// api_diff.cu, api_batch.cu and api_extra.cu; shared helpers in ctx.cu.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "context.cuh"

using namespace scgr;
using namespace scgr::api;

namespace {
thread_local std::string g_create_error;
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
                    &c->bcpair, &c->btabX, &c->btabY, &c->bxoff, &c->byoff, &c->bstats, &c->bposes, &c->bnext,
                    &c->gcell, &c->gcount, &c->gstart, &c->gcursor, &c->gblock, &c->gsorted, &c->gsidx, &c->gbb,
                    &c->rgstart, &c->rgsorted, &c->rgsidx, &c->rcgstart, &c->rcgsorted, &c->rcgsidx,
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
  NvtxRange nvtx_range("scgr_compute_descriptors");
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
  NvtxRange nvtx_range("scgr_run");
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
      c->graph_launches = c->launches - before;  // kernel launches in the graph, counted at each replay
      c->launches = before;
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
    c->launches += c->graph_launches;
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
  NvtxRange nvtx_range("scgr_forces");
  if (!c || !f4_dev) return fail(c, SCGR_ERR_INVALID_ARG, "NULL argument");
  c->err.clear();
  if (!c->have_desc) return fail(c, SCGR_ERR_STATE, "compute descriptors first");
  scgr_status fs = force_launch(c);
  if (fs != SCGR_OK) return fs;
  const int mloc = (int)(c->rows >= 0 ? c->rows : c->m);
  SCGR_CK(c, launch_combine(c->L(), (const float4*)c->partial.p, c->fp.splits, (int)c->mpad, mloc,
                            (const float4*)c->Y0r.p, (const float*)c->aY32.p + c->row0, c->prm.g_mode, c->pose,
                            (float4*)f4_dev, (double*)c->blockpart.p));
  return SCGR_OK;
}

scgr_status scgr_set_curvature(scgr_ctx* c, int which, const double* a64_dev) {
  NvtxRange nvtx_range("scgr_set_curvature");
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

scgr_status scgr_plan_preview(int64_t n, int64_t m, double p, int num_sms, int blocks_per_sm, int out[7]) {
  if (!out || n < 1 || m < 1 || !(p >= 1.0) || !std::isfinite(p) || num_sms < 1 || blocks_per_sm < 1)
    return SCGR_ERR_INVALID_ARG;
  const int64_t npad = (n + FORCE_TJ - 1) / FORCE_TJ * FORCE_TJ;
  const ForcePlan fp = plan_force(m, npad, p, num_sms, ForceTuning(), blocks_per_sm);
  out[0] = fp.P;
  out[1] = fp.tpb;
  out[2] = fp.occ;
  out[3] = fp.splits;
  out[4] = fp.tiles_per_split;
  out[5] = fp.iblocks;
  out[6] = fp.half;
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
    if (value < 0 || value > 2) return fail(c, SCGR_ERR_INVALID_ARG, "occupancy variant must be 0, 1 or 2");
    c->ftune.occ = value;
    return c->have_desc ? replan(c) : SCGR_OK;
  }
  if (key == SCGR_TUNE_FORCE_SPLITS) {
    if (value < 0 || value > 4096) return fail(c, SCGR_ERR_INVALID_ARG, "splits must be in [0, 4096]");
    c->ftune.splits = value;
    return c->have_desc ? replan(c) : SCGR_OK;
  }
  if (key == SCGR_TUNE_FORCE_RSQRT) {
    if (value < 0 || value > 2) return fail(c, SCGR_ERR_INVALID_ARG, "distance factor form must be 0, 1 or 2");
    c->ftune.rsq = value;
    return c->have_desc ? replan(c) : SCGR_OK;
  }
  if (key == SCGR_TUNE_FORCE_EX2POLY) {
    if (value < 0 || value > 2) return fail(c, SCGR_ERR_INVALID_ARG, "value must be 0, 1 or 2");
    c->ftune.ex2poly = value;
    return c->have_desc ? replan(c) : SCGR_OK;
  }
  if (key == SCGR_TUNE_NEAREST_LEVELS) {
    if (value != 1 && value != 2) return fail(c, SCGR_ERR_INVALID_ARG, "value must be 1 or 2");
    c->nearest_levels = value;
    return SCGR_OK;
  }
  if (key == SCGR_TUNE_FUSED_TAIL) {
    if (value != 0 && value != 1) return fail(c, SCGR_ERR_INVALID_ARG, "value must be 0 or 1");
    c->fused_tail = value;
    drop_graph(c);
    return SCGR_OK;
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
  if (key == SCGR_TUNE_NEAREST_GRID_MIN) {
    if (value < 0) return fail(c, SCGR_ERR_INVALID_ARG, "grid threshold must be >= 0");
    c->nearest_grid_min = value;
    return SCGR_OK;
  }
  if (key == SCGR_TUNE_BATCH_P) {
    if (value != 0 && value != 1 && value != 2 && value != 4)
      return fail(c, SCGR_ERR_INVALID_ARG, "batch points per thread must be 0 (mixed), 1, 2 or 4");
    c->batch_P = value;
    return SCGR_OK;
  }
  if (key == SCGR_TUNE_BATCH_PERSISTENT) {
    if (value != 0 && value != 1) return fail(c, SCGR_ERR_INVALID_ARG, "value must be 0 or 1");
    c->batch_persistent = value;
    return SCGR_OK;
  }
  if (key == SCGR_TUNE_BATCH_CHUNK_TILES) {
    if (value < 1 || value > 4096) return fail(c, SCGR_ERR_INVALID_ARG, "chunk tiles must be in [1, 4096]");
    c->batch_chunk_tiles = value;
    return SCGR_OK;
  }
  return fail(c, SCGR_ERR_INVALID_ARG, "unknown tuning key");
}

int64_t scgr_launch_count(const scgr_ctx* c) { return c ? c->launches : -1; }

scgr_status scgr_debug_fail_allocations(int count) {
  if (count < 0) return SCGR_ERR_INVALID_ARG;
  g_fail_allocs.store(count);
  return SCGR_OK;
}

}  // extern "C"
