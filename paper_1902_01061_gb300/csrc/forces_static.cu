// scgr_forces_static: the per-point force evaluation (Eq. 5) for callers that
// cannot allocate device memory.
//
// Who needs it: hosts whose device memory is fully owned by another allocator
// (a framework's caching pool, a fixed budget on an embedded robot), and
// tight real-time loops (e.g. the paper's Kinect change-detection setting)
// that cannot take cudaMalloc's latency or the device-wide synchronisation a
// cudaFree can cause.  Such callers cannot create a context, because a
// context allocates its workspace.  This entry point takes the clouds,
// curvatures and output from the caller and keeps every intermediate buffer
// in one file-scope __device__ array of fixed size (STATIC_BYTES, about
// 25 MB).  Every GPU that loads the library holds that array until the
// process exits.
//
// It reuses the library's kernels unchanged (pack, statistics, sigma, force
// records, the all-pairs force kernel and the combine); only the pointers
// differ, and the reference range is split at most STATIC_MAX_SPLITS ways so
// that the per-split partial sums fit.
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>

#include "common.cuh"
#include "scgr.h"

namespace scgr {
namespace {

constexpr int64_t STATIC_MAX_POINTS = 131072;  // per cloud
constexpr int STATIC_MAX_SPLITS = 8;
constexpr int64_t STATIC_MPAD_MAX = STATIC_MAX_POINTS + 1024;

constexpr size_t al256(size_t x) { return (x + 255) / 256 * 256; }
constexpr size_t OFF_X4 = 0;
constexpr size_t OFF_Y4 = OFF_X4 + al256(16 * STATIC_MAX_POINTS);
constexpr size_t OFF_XR = OFF_Y4 + al256(16 * STATIC_MAX_POINTS);
constexpr size_t OFF_XA = OFF_XR + al256(16 * STATIC_MAX_POINTS);
constexpr size_t OFF_Y0R = OFF_XA + al256(8 * STATIC_MAX_POINTS);
constexpr size_t OFF_PART = OFF_Y0R + al256(16 * STATIC_MPAD_MAX);
constexpr size_t OFF_BLK = OFF_PART + al256(16 * STATIC_MAX_SPLITS * STATIC_MPAD_MAX);
constexpr size_t OFF_RED = OFF_BLK + al256(8 * 13 * (STATIC_MPAD_MAX / 256 + 1));
constexpr size_t OFF_A32X = OFF_RED + al256(8 * (RED_MAX_BLOCKS * 6 + 32));
constexpr size_t OFF_A32Y = OFF_A32X + al256(4 * STATIC_MAX_POINTS);
constexpr size_t OFF_STATS = OFF_A32Y + al256(4 * STATIC_MAX_POINTS);
constexpr size_t OFF_POSE = OFF_STATS + al256(sizeof(DevStats));
constexpr size_t OFF_ERR = OFF_POSE + al256(sizeof(DevPose));
constexpr size_t STATIC_BYTES = OFF_ERR + 256;

}  // namespace
}  // namespace scgr

// The shared scratch.  In host code this name is only a stand-in: kernels get
// the device address that cudaGetSymbolAddress returns for the current device.
static __device__ __align__(256) unsigned char g_forces_scratch[scgr::STATIC_BYTES];

namespace {

constexpr int MAX_DEVICES = 64;
std::mutex g_setup_mutex;
unsigned char* g_scratch_addr[MAX_DEVICES] = {nullptr};
int g_num_sms[MAX_DEVICES] = {0};

// Device address of the scratch on the current device, looked up once per
// device (with that device current).
cudaError_t scratch_for_current_device(unsigned char** out, int* num_sms) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= MAX_DEVICES) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_forces_scratch);
    if (e != cudaSuccess) return e;
    int sms = 0;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    g_scratch_addr[dev] = static_cast<unsigned char*>(p);
    g_num_sms[dev] = sms;
  }
  *out = g_scratch_addr[dev];
  *num_sms = g_num_sms[dev];
  return cudaSuccess;
}

}  // namespace

extern "C" scgr_status scgr_forces_static(const float* x_dev, int64_t n, const float* y_dev, int64_t m,
                                          const double* ax_dev, const double* ay_dev, double sigma,
                                          double p, int g_mode, float* f4_dev, void* cuda_stream) {
  using namespace scgr;
  if (!x_dev || !y_dev || !ax_dev || !ay_dev || !f4_dev) return SCGR_ERR_INVALID_ARG;
  if (n < 1 || m < 1 || n > STATIC_MAX_POINTS || m > STATIC_MAX_POINTS) return SCGR_ERR_INVALID_ARG;
  if (!(p >= 1.0) || !std::isfinite(p) || !std::isfinite(sigma)) return SCGR_ERR_INVALID_ARG;
  if (g_mode != 0 && g_mode != 1) return SCGR_ERR_INVALID_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);

  unsigned char* base = nullptr;
  int num_sms = 0;
  if (scratch_for_current_device(&base, &num_sms) != cudaSuccess) {
    cudaGetLastError();
    return SCGR_ERR_CUDA;
  }
  float4* X4 = reinterpret_cast<float4*>(base + OFF_X4);
  float4* Y4 = reinterpret_cast<float4*>(base + OFF_Y4);
  float4* Xr = reinterpret_cast<float4*>(base + OFF_XR);
  float2* XA = reinterpret_cast<float2*>(base + OFF_XA);
  float4* Y0r = reinterpret_cast<float4*>(base + OFF_Y0R);
  float4* partial = reinterpret_cast<float4*>(base + OFF_PART);
  double* blockpart = reinterpret_cast<double*>(base + OFF_BLK);
  double* red = reinterpret_cast<double*>(base + OFF_RED);
  float* a32x = reinterpret_cast<float*>(base + OFF_A32X);
  float* a32y = reinterpret_cast<float*>(base + OFF_A32Y);
  DevStats* stats = reinterpret_cast<DevStats*>(base + OFF_STATS);
  DevPose* pose = reinterpret_cast<DevPose*>(base + OFF_POSE);
  int* err = reinterpret_cast<int*>(base + OFF_ERR);

  const int64_t npad = (n + 255) / 256 * 256;
  ForcePlan fp = plan_force(m, npad, p, num_sms);
  const int ntiles = (int)(npad / fp.tile_j);
  if (fp.splits > STATIC_MAX_SPLITS) {
    fp.half = 0;
    const int sub = force_stage_tiles(fp);
    fp.tiles_per_split = ((ntiles + STATIC_MAX_SPLITS - 1) / STATIC_MAX_SPLITS + sub - 1) / sub * sub;
    fp.splits = (ntiles + fp.tiles_per_split - 1) / fp.tiles_per_split;
  }
  const int64_t mpad = force_mpad(m, fp);
  if (mpad > STATIC_MPAD_MAX || fp.splits > STATIC_MAX_SPLITS) return SCGR_ERR_INVALID_ARG;

  Launch L{st, nullptr};
  cudaError_t e = cudaMemsetAsync(err, 0, sizeof(int), st);  // the error word must start at zero
  if (e == cudaSuccess) e = launch_pack(L, x_dev, n, X4, err);
  if (e == cudaSuccess) e = launch_pack(L, y_dev, m, Y4, err);
  if (e == cudaSuccess) e = launch_check_curvature(L, ax_dev, (int)n, a32x, err);
  if (e == cudaSuccess) e = launch_check_curvature(L, ay_dev, (int)m, a32y, err);
  if (e == cudaSuccess) e = launch_cloud_stats(L, X4, (int)n, red, stats->xbar, stats->CX, &stats->eX);
  if (e == cudaSuccess) e = launch_cloud_stats(L, Y4, (int)m, red, stats->ybar0, stats->S0, &stats->eY0);
  if (e == cudaSuccess) e = launch_sigma(L, ax_dev, (int)n, sigma, red, &stats->sigma, &stats->asum[0]);
  if (e == cudaSuccess)
    e = launch_records(L, X4, ax_dev, (int)n, (int)npad, Y4, ay_dev, (int)m, (int)mpad, g_mode, stats, Xr, XA, Y0r);
  if (e == cudaSuccess) e = launch_pose_init(L, pose, stats, 1);
  if (e == cudaSuccess)
    e = launch_force(L, fp, Xr, XA, ntiles, Y0r, (int)mpad, pose, (float)((p - 1.0) * 0.5), partial);
  if (e == cudaSuccess) e = launch_combine(L, partial, fp.splits, (int)mpad, (int)m, Y0r, a32y, g_mode, pose, reinterpret_cast<float4*>(f4_dev), blockpart);
  int herr = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return e == cudaErrorMemoryAllocation ? SCGR_ERR_OOM : SCGR_ERR_CUDA;
  }
  if (herr & ERR_NONFINITE) return SCGR_ERR_NONFINITE;
  return SCGR_OK;
}
