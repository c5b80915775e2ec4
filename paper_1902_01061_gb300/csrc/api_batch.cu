// C ABI, batching form: many registrations of uneven sizes in one call.
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

scgr_status scgr_batch_run(scgr_ctx* c, int npairs, const int64_t* ref_off, const float* ref_xyz_dev,
                           const int64_t* tmp_off, const float* tmp_xyz_dev, int iterations,
                           scgr_result* results) {
  NvtxRange nvtx_range("scgr_batch_run");
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
  const bool mixed = c->batch_P == 0;  // per-pair shape: 4 x 128 (512-point blocks) or 2 x 128 (256)
  const int FB0 = mixed ? 256 : batch_block_threads(c->batch_P) * c->batch_P;  // template points per force block
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
    bp.shape4 = mixed && batch_pair_shape4(bp.m) ? 1 : 0;
    const int FB = bp.shape4 ? 512 : FB0;
    bp.xtile0 = xt;
    xt += bp.ntiles;
    const int64_t round = FB > 256 ? FB : 256;  // whole force blocks and combine blocks
    bp.mpad = (bp.m + round - 1) / round * round;
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
  // kNN blocks scan their whole cloud: biggest clouds first, so the small
  // ones fill the last wave
  std::stable_sort(tabX.begin(), tabX.end(), [&](const int2& a, const int2& b) { return pairs[a.x].n > pairs[b.x].n; });
  std::stable_sort(tabY.begin(), tabY.end(), [&](const int2& a, const int2& b) { return pairs[a.x].m > pairs[b.x].m; });
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
  SCGR_CK(c, ensure(c->bnext, sizeof(int)));
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
  const int pmode = (c->prm.p == 1.0) ? 1 : (c->prm.p == 2.0) ? (c->ftune.rsq == 1 ? 4 : 2) : (c->prm.p == 3.0) ? 3 : 0;
  int pgrid = 0;  // persistent form: one resident block per slot (queried before any capture)
  if (c->batch_persistent && !mixed) SCGR_CK(c, force_batch_slots(pmode, c->batch_P, &pgrid));
  auto enqueue = [&](Launch LL) -> scgr_status {
    for (int t = 0; t < iterations; ++t) {
      SCGR_CK(c, launch_force_batch(LL, pmode, c->batch_P, (int)items.size(), (const int4*)c->bitems.p, dpairs,
                                    (const float4*)c->bXr.p, (const float2*)c->bXA.p, (const float4*)c->bY0r.p,
                                    (const DevPose*)c->bposes.p, c->qexp, (float4*)c->bpartial.p, CT, pgrid,
                                    (int*)c->bnext.p));
      SCGR_CK(c, launch_combine_batch(LL, cb, (const int*)c->bcpair.p, dpairs, (const float4*)c->bpartial.p,
                                      (const float4*)c->bY0r.p, (const float*)c->baY32.p, c->prm.g_mode,
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
      const int64_t in_graph = c->launches - before;  // kernel launches of the graph, counted at its replay
      c->launches = before;
      if (stq != SCGR_OK) { if (g) cudaGraphDestroy(g); return stq; }
      if (e != cudaSuccess) return cuda_fail(c, e, "batch graph capture");
      c->bgraph = g;
      SCGR_CK(c, cudaGraphInstantiate(&c->bgexec, c->bgraph, 0));
      SCGR_CK(c, cudaGraphLaunch(c->bgexec, c->cap_stream));
      SCGR_CK(c, cudaEventRecord(c->join_out, c->cap_stream));
      SCGR_CK(c, cudaStreamWaitEvent(c->stream, c->join_out, 0));
      c->launches += in_graph;
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

}  // extern "C"
