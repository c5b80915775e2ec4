// C ABI, differentiation form: the shape-weighted potential, its adjoint
// (recomputed tiles or stored pair terms) and the force-field VJP.
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

scgr_status scgr_potential(scgr_ctx* c, const double pose7[7], double* U_out, double* grad_pose7,
                           float* grad_xyz_dev) {
  NvtxRange nvtx_range("scgr_potential");
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
                            (const float4*)c->Y0r.p, (const float*)c->aY32.p, c->prm.g_mode, c->pose_eval,
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

scgr_status scgr_potential_stored(scgr_ctx* c, const double pose7[7], double* U_out, double* grad_pose7,
                                  float* grad_xyz_dev) {
  NvtxRange nvtx_range("scgr_potential_stored");
  if (!c || !pose7 || !U_out) return fail(c, SCGR_ERR_INVALID_ARG, "NULL argument");
  c->err.clear();
  if (!c->have_desc) return fail(c, SCGR_ERR_STATE, "compute descriptors first");
  if (c->rows >= 0) return fail(c, SCGR_ERR_STATE, "the potential needs the whole template (a row range is set)");
  for (int q = 0; q < 7; ++q)
    if (!std::isfinite(pose7[q])) return fail(c, SCGR_ERR_INVALID_ARG, "non-finite pose");
  if (!(pose7[6] > 0.0)) return fail(c, SCGR_ERR_INVALID_ARG, "scale must be > 0");
  const int npad = (int)c->npad, m = (int)c->m;
  SCGR_CK(c, ensure(c->wstore, (size_t)npad * m * sizeof(float)));
  SCGR_CK(c, ensure(c->wupart, (size_t)store_pairs_columns(npad) * store_pairs_row_blocks(m) * sizeof(double)));
  SCGR_CK(c, ensure(c->wpartial, (size_t)c->mpad * sizeof(float4)));
  Launch L = c->L();
  double* d7 = c->aux + 48;
  SCGR_CK(c, cudaMemcpyAsync(d7, pose7, 7 * sizeof(double), cudaMemcpyHostToDevice, c->stream));
  SCGR_CK(c, launch_pose_from7(L, d7, c->pose_eval, c->stats));
  // forward: store w_ij and sum U
  SCGR_CK(c, launch_store_pairs(L, (const float2*)c->XA.p, (const float4*)c->Xr.p, npad, (const float4*)c->Y0r.p,
                                (const double*)c->aY64.p, c->prm.g_mode, m, c->pose_eval, c->qexp,
                                (float*)c->wstore.p, (double*)c->wupart.p, c->aux + 3));
  if (grad_pose7 || grad_xyz_dev) {
    // backward from the stored terms
    SCGR_CK(c, launch_stored_rows(L, (const float*)c->wstore.p, npad, m, (const float4*)c->Xr.p,
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
  NvtxRange nvtx_range("scgr_force_vjp");
  if (!c || !v_dev || !grad_dev) return fail(c, SCGR_ERR_INVALID_ARG, "NULL argument");
  c->err.clear();
  if (!c->have_desc) return fail(c, SCGR_ERR_STATE, "compute descriptors first");
  if (c->rows >= 0) return fail(c, SCGR_ERR_STATE, "the VJP needs the whole template (a row range is set)");
  SCGR_CK(c, launch_force_vjp(c->L(), (const float4*)c->Xr.p, (const float2*)c->XA.p, (int)(c->npad / FORCE_TJ),
                              (const float4*)c->Y0r.p, (const double*)c->aY64.p, c->prm.g_mode, (int)c->m, c->pose,
                              c->prm.p, v_dev, grad_dev));
  return SCGR_OK;
}

}  // extern "C"
