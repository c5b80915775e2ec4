// Internal: the scgr_ctx context (device workspace, plan, pose, graphs) and
// the helpers the entry-point files share.  Not part of the C ABI.
#pragma once
#include <cuda_runtime.h>

#include <atomic>
#include <cstdint>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "common.cuh"
#include "scgr.h"

namespace scgr {
namespace api {

// NVTX range for the duration of a scope (stages show up in profiler
// timelines; free when no profiler is attached).
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

// A device buffer that grows on demand.
struct DevBuf {
  void* p = nullptr;
  size_t cap = 0;
};

}  // namespace api
}  // namespace scgr

using scgr::api::DevBuf;
using scgr::DevPose;
using scgr::DevStats;
using scgr::ForcePlan;
using scgr::ForceTuning;
using scgr::Launch;
using scgr::GridSpec;

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
  int64_t graph_launches = 0;  // kernel launches one replay of the graph makes
  bool capturing = false;
  cudaStream_t cap_stream = nullptr;  // capture / replay stream (never the legacy stream)
  cudaEvent_t join_in = nullptr, join_out = nullptr;

  // batch workspace
  DevBuf bX4, bY4, bknnX, bknnY, baX64, baY64, baX32, baY32, bXr, bXA, bY0r, bpartial, bblockpart,
      bpairs, bitems, bcpair, btabX, btabY, bxoff, byoff, bstats, bposes, bnext;
  int batch_chunk_tiles = 16;   // reference tiles per batched work item (tunable)
  int batch_P = 1;              // template points per thread in the batched force kernel (tunable)
  int batch_persistent = 0;     // 1: persistent batched force kernel with a work queue (tunable)
  int64_t knn_grid_min = 20000; // clouds with at least this many points use the grid kNN (tunable)
  int64_t nearest_grid_min = 65536; // references with at least this many points: grid nearest search (tunable)
  ForceTuning ftune;            // force-plan overrides (tunable)
  int reuse_pose_free = 1;      // p = 1: one force pass per scgr_run (tunable)
  DevBuf gcell, gcount, gstart, gcursor, gblock, gsorted, gsidx, gbb, cd_key, cd_moved, wstore, wupart, wpartial,
      mpart, mom;
  // the reference's grid for nearest-point queries, kept until the reference changes
  DevBuf rgstart, rgsorted, rgsidx, rcgstart, rcgsorted, rcgsidx;  // fine and coarse levels
  GridSpec rgspec{}, rcgspec{};
  bool rgrid_ok = false;
  int nearest_levels = 2;       // 2: two-level nearest search (default), 1: fine shells only (tunable)
  int fused_tail = 1;           // 1: one combine-finalize launch for small templates (tunable)
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

namespace scgr {
namespace api {

scgr_status fail(scgr_ctx* c, scgr_status st, const std::string& msg);
scgr_status cuda_fail(scgr_ctx* c, cudaError_t e, const char* where);

// Return a CUDA failure of `call` as SCGR_ERR_CUDA / SCGR_ERR_OOM with its text.
#define SCGR_CK(ctx, call)                                              \
  do {                                                                  \
    cudaError_t e_ = (call);                                            \
    if (e_ != cudaSuccess) return scgr::api::cuda_fail(ctx, e_, #call); \
  } while (0)

cudaError_t ensure(DevBuf& b, size_t bytes);
extern std::atomic<int> g_fail_allocs;
void release(DevBuf& b);
scgr_status check_params(const scgr_params* p, std::string& why);
StepParams step_params(const scgr_ctx* c);
scgr_status read_error_word(scgr_ctx* c);
scgr_status set_cloud(scgr_ctx* c, const float* xyz, int64_t n, bool host, bool ref);
scgr_status force_launch(scgr_ctx* c);
scgr_status collect_timing(scgr_ctx* c);
scgr_status knn_cloud(scgr_ctx* c, const float4* P, int n, int32_t* out);
scgr_status nearest_reference(scgr_ctx* c, const float* q3, int nq, int32_t* idx_out, float* key_out);
scgr_status curvatures(scgr_ctx* c, int k, double radius_scale, double sigma_scale);
scgr_status replan(scgr_ctx* c);
scgr_status enqueue_iterations(scgr_ctx* c, int iters);
void drop_graph(scgr_ctx* c);

}  // namespace api
}  // namespace scgr
