// C ABI, neighbourhood schedule, change detection and template-row sharding.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "context.cuh"

using namespace scgr;
using namespace scgr::api;

extern "C" {

scgr_status scgr_nearest(scgr_ctx* c, const float* q_dev, int64_t nq, int32_t* idx_dev, float* key_dev) {
  if (!c || !q_dev || (!idx_dev && !key_dev)) return fail(c, SCGR_ERR_INVALID_ARG, "NULL argument");
  c->err.clear();
  if (!c->have_X) return fail(c, SCGR_ERR_STATE, "set the reference first");
  if (nq < 0 || nq > (int64_t(1) << 30)) return fail(c, SCGR_ERR_INVALID_ARG, "bad query count");
  return nearest_reference(c, q_dev, (int)nq, idx_dev, key_dev);
}

scgr_status scgr_change_mask(scgr_ctx* c, double threshold, uint8_t* mask_dev, float* dist_dev) {
  NvtxRange nvtx_range("scgr_change_mask");
  if (!c || !mask_dev) return fail(c, SCGR_ERR_INVALID_ARG, "NULL argument");
  c->err.clear();
  if (!c->have_desc) return fail(c, SCGR_ERR_STATE, "compute descriptors first");
  if (!(threshold >= 0.0) || !std::isfinite(threshold)) return fail(c, SCGR_ERR_INVALID_ARG, "threshold must be >= 0");
  const int m = (int)c->m;
  SCGR_CK(c, ensure(c->cd_moved, (size_t)m * 3 * sizeof(float)));
  SCGR_CK(c, ensure(c->cd_key, (size_t)m * sizeof(float)));
  SCGR_CK(c, launch_apply(c->L(), (const float4*)c->Y4.p, m, c->pose, (float*)c->cd_moved.p));
  const scgr_status st = nearest_reference(c, (const float*)c->cd_moved.p, m, nullptr, (float*)c->cd_key.p);
  if (st != SCGR_OK) return st;
  SCGR_CK(c, launch_threshold(c->L(), (const float*)c->cd_key.p, m, (float)(threshold * threshold), mask_dev,
                              dist_dev));
  return SCGR_OK;
}

scgr_status scgr_set_neighbourhood(scgr_ctx* c, int k, double radius_scale, double sigma_scale) {
  NvtxRange nvtx_range("scgr_set_neighbourhood");
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
  NvtxRange nvtx_range("scgr_step_partials");
  if (!c || !out13) return fail(c, SCGR_ERR_INVALID_ARG, "NULL argument");
  c->err.clear();
  if (!c->have_desc) return fail(c, SCGR_ERR_STATE, "compute descriptors first");
  if (c->E_host <= 0) return fail(c, SCGR_ERR_STATE, "set params.E for stepwise iteration");
  const int mloc = (int)(c->rows >= 0 ? c->rows : c->m);
  scgr_status fs = force_launch(c);
  if (fs != SCGR_OK) return fs;
  SCGR_CK(c, launch_combine(c->L(), (const float4*)c->partial.p, c->fp.splits, (int)c->mpad, mloc,
                            (const float4*)c->Y0r.p, (const float*)c->aY32.p + c->row0, c->prm.g_mode, c->pose,
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

// Stream-ordered forms of the two halves of a sharded iteration: nothing is
// copied to or from the host and nothing waits, so the exchange between them
// can be a collective enqueued on the same stream (an NCCL all-gather) and a
// run of iterations never leaves the device.
scgr_status scgr_step_partials_dev(scgr_ctx* c, double* out13_dev) {
  NvtxRange nvtx_range("scgr_step_partials_dev");
  if (!c || !out13_dev) return fail(c, SCGR_ERR_INVALID_ARG, "NULL argument");
  c->err.clear();
  if (!c->have_desc) return fail(c, SCGR_ERR_STATE, "compute descriptors first");
  if (c->E_host <= 0) return fail(c, SCGR_ERR_STATE, "set params.E for stepwise iteration");
  const int mloc = (int)(c->rows >= 0 ? c->rows : c->m);
  scgr_status fs = force_launch(c);
  if (fs != SCGR_OK) return fs;
  SCGR_CK(c, launch_combine(c->L(), (const float4*)c->partial.p, c->fp.splits, (int)c->mpad, mloc,
                            (const float4*)c->Y0r.p, (const float*)c->aY32.p + c->row0, c->prm.g_mode, c->pose,
                            nullptr, (double*)c->blockpart.p));
  SCGR_CK(c, launch_column_sum13(c->L(), (const double*)c->blockpart.p, combine_blocks(c->mpad), out13_dev));
  return SCGR_OK;
}

scgr_status scgr_step_apply_dev(scgr_ctx* c, const double* parts_dev, int nparts) {
  NvtxRange nvtx_range("scgr_step_apply_dev");
  if (!c || !parts_dev) return fail(c, SCGR_ERR_INVALID_ARG, "NULL argument");
  c->err.clear();
  if (nparts < 1 || nparts > 65536) return fail(c, SCGR_ERR_INVALID_ARG, "nparts must be in [1, 65536]");
  if (!c->have_desc) return fail(c, SCGR_ERR_STATE, "compute descriptors first");
  if (c->E_host <= 0) return fail(c, SCGR_ERR_STATE, "set params.E for stepwise iteration");
  SCGR_CK(c, launch_finalize(c->L(), parts_dev, nparts, c->pose, c->stats, step_params(c), c->errword));
  c->iterations += 1;
  return SCGR_OK;
}

}  // extern "C"
