// Shared device-side declarations of the scgr CUDA library (sm_103a).
//
// Data layout in HBM (one context):
//   X4, Y4      float4 [n] packed input clouds (x, y, z, 0), original frame
//   knnX, knnY  int32 [n][k] neighbour lists sorted by (key, index)
//   aX64, aY64  float64 [n] curvature (Sec. III-A), aX32/aY32 float32 copies
//   Xr          float [npad/TJ][4][TJ] force-kernel reference records, tile-major
//               structure-of-arrays: x', y', z' (frame centred on the reference
//               mean) and |X'|^2 for each tile of FORCE_TJ points
//   XA          float [npad/TJ][2][TJ]: a_hat = a * sqrt(log2 e) / sigma and
//               -L (L = log2 aX, or 0 in the mode g = s)
//   Y0r         float4 [mpad] (Y0x, Y0y, Y0z, a_hat) template record
//   partial     float4 [S][mpad] per-split (sum w, sum w X') of the force kernel
//   blockpart   float64 [nblocks][13] per-block (F, W, T) of the combine kernel
//   pose/stats  small float64 structs below
#pragma once
#include <cuda_runtime.h>
#include <cstdint>

namespace scgr {

constexpr int ERR_NONFINITE = 1;
constexpr int ERR_NUMERIC = 2;
constexpr int ERR_TIMEOUT = 4;

// Iteration state kept on the device so that the whole loop runs without a
// host round trip (and can be captured in a CUDA graph).
struct DevPose {
  double R[9];     // row-major, row-vector convention: Y = s Y0 R + t
  double t[3];
  double s;
  double ybs[3];   // template mean minus reference mean at this pose
  float A[9];      // float32 map used by the force kernel: Y' = Y0 A + b
  float b[3];      //   with A = s R and b = t - xbar (frame centred on xbar)
  float ych[3];    // ybs as a float pair ych + ycl, read by the per-point
  float ycl[3];    //   combine kernels (set together with ybs by set_ybs)
  int it;          // next iteration index of Eq. 12
  int E;           // Eq. 12 horizon
  int degenerate;  // iterations with a rank < 2 cross-covariance
  int pad;
};

// ybs[c] = v and its float pair (ych + ycl = v to about 2^-48 relative).
__device__ __forceinline__ void set_ybs(DevPose* ps, int c, double v) {
  ps->ybs[c] = v;
  const float h = (float)v;
  ps->ych[c] = h;
  ps->ycl[c] = (float)(v - (double)h);
}

// Cloud statistics of the scale model (Sec. III-B) and sigma of Eq. 3.
struct DevStats {
  double xbar[3];
  double CX[9];    // scatter sum_j (X_j - xbar)^T (X_j - xbar), unnormalised
  double eX;       // largest eigenvalue of CX / N
  double ybar0[3];
  double S0[9];    // scatter sum_i (Y0_i - ybar0)^T (Y0_i - ybar0), unnormalised
  double eY0;      // largest eigenvalue of S0 / M
  double sigma;
  double asum[2];  // sum of curvatures of X, Y0 (diagnostic)
};

// Method constants the finalize kernel needs (passed by value).
struct StepParams {
  double G1, eta0, time;
  int step_mode, scale_mode;
  int M;
};

// ---- fixed-order float64 reductions ------------------------------------
constexpr int RED_THREADS = 256;
constexpr int RED_MAX_BLOCKS = 1024;

inline int red_blocks(int64_t n) {
  int64_t b = (n + RED_THREADS - 1) / RED_THREADS;
  if (b < 1) b = 1;
  if (b > RED_MAX_BLOCKS) b = RED_MAX_BLOCKS;
  return (int)b;
}

// Sum v[0..NV) over the block in a fixed tree order; thread 0 gets the result.
template <int NV>
__device__ __forceinline__ void block_sum(double (&v)[NV], double (*sh)[RED_THREADS]) {
  const int t = threadIdx.x;
#pragma unroll
  for (int q = 0; q < NV; ++q) sh[q][t] = v[q];
  __syncthreads();
  for (int w = RED_THREADS / 2; w > 0; w >>= 1) {
    if (t < w) {
#pragma unroll
      for (int q = 0; q < NV; ++q) sh[q][t] += sh[q][t + w];
    }
    __syncthreads();
  }
#pragma unroll
  for (int q = 0; q < NV; ++q) v[q] = sh[q][0];
}

// Packed FP32 pairs (Blackwell add/sub/mul/fma .f32x2): each instruction
// works on two float32 lanes with the same per-lane IEEE rounding as the
// scalar .rn instruction (no contraction, subnormals kept).
typedef unsigned long long u64;  // two packed float32 lanes (low, high)

__device__ __forceinline__ u64 pk2(float lo, float hi) {
  u64 r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
  return r;
}
__device__ __forceinline__ void upk2(u64 v, float& lo, float& hi) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
__device__ __forceinline__ u64 add2(u64 a, u64 b) {
  u64 d;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ u64 sub2(u64 a, u64 b) {
  u64 d;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ u64 mul2(u64 a, u64 b) {
  u64 d;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ u64 fma2(u64 a, u64 b, u64 c) {
  u64 d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}
// Symmetric 3x3 eigenvalues by cyclic Jacobi rotations (float64), ascending.
__host__ __device__ inline void sym3_eigenvalues(const double* Ain, double* lam) {
  double a[3][3];
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c) a[r][c] = 0.5 * (Ain[r * 3 + c] + Ain[c * 3 + r]);
  for (int sweep = 0; sweep < 32; ++sweep) {
    const double off = a[0][1] * a[0][1] + a[0][2] * a[0][2] + a[1][2] * a[1][2];
    const double dia = a[0][0] * a[0][0] + a[1][1] * a[1][1] + a[2][2] * a[2][2];
    if (off <= 1e-36 * dia || off == 0.0) break;
    for (int pq = 0; pq < 3; ++pq) {
      const int p = pq == 2 ? 1 : 0;
      const int q = pq == 0 ? 1 : 2;
      const double apq = a[p][q];
      if (apq == 0.0) continue;
      const double theta = (a[q][q] - a[p][p]) / (2.0 * apq);
      double t;
      if (fabs(theta) > 1e150) t = 0.5 / theta;
      else t = (theta >= 0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
      const double c = 1.0 / sqrt(t * t + 1.0);
      const double s = t * c;
      const int r = 3 - p - q;
      const double arp = a[r][p], arq = a[r][q];
      a[p][p] -= t * apq;
      a[q][q] += t * apq;
      a[p][q] = a[q][p] = 0.0;
      a[r][p] = a[p][r] = c * arp - s * arq;
      a[r][q] = a[q][r] = s * arp + c * arq;
    }
  }
  double l0 = a[0][0], l1 = a[1][1], l2 = a[2][2], tmp;
  if (l0 > l1) { tmp = l0; l0 = l1; l1 = tmp; }
  if (l1 > l2) { tmp = l1; l1 = l2; l2 = tmp; }
  if (l0 > l1) { tmp = l0; l0 = l1; l1 = tmp; }
  lam[0] = l0; lam[1] = l1; lam[2] = l2;
}

// Smallest eigenvalue of a symmetric positive semi-definite 3x3 C (row-major)
// as the smallest root of its characteristic polynomial
//   f(l) = det(C - l I) = p0 - p1 l + p2 l^2 - l^3
// by Newton's method from l = 0.  On [0, l_min] f is positive, decreasing and
// convex, so the iterates rise monotonically to l_min with no overshoot
// (quadratically for a simple root).  A few FP64 steps replace the sweeps of
// Jacobi rotations, each with square roots and divisions.  Where the root is
// (nearly) multiple, Newton slows down and f near the root is lost in
// rounding, so after 12 steps, or when f reaches its rounding level without
// a quadratic last step, the Jacobi solver takes over.
// Returns 0 when C is singular to rounding (f(0) <= 0 or p1 = 0).
__host__ __device__ inline double sym3_min_eigenvalue(const double* C) {
  const double c00 = C[0], c11 = C[4], c22 = C[8];
  const double c01 = 0.5 * (C[1] + C[3]), c02 = 0.5 * (C[2] + C[6]), c12 = 0.5 * (C[5] + C[7]);
  const double p2 = c00 + c11 + c22;
  const double m00 = c11 * c22 - c12 * c12, m11 = c00 * c22 - c02 * c02, m22 = c00 * c11 - c01 * c01;
  const double p1 = m00 + m11 + m22;
  const double p0 = c00 * m00 - c01 * (c01 * c22 - c12 * c02) + c02 * (c01 * c12 - c11 * c02);
  if (!(p0 > 0.0) || !(p1 > 0.0)) return 0.0;
  double l = 0.0, last = p2;
  for (int it = 0; it < 12; ++it) {
    const double f = p0 + l * (-p1 + l * (p2 - l));
    const double df = -p1 + l * (2.0 * p2 - 3.0 * l);
    if (!(f > 0.0) || !(df < 0.0)) {  // f is at its rounding level
      if (last <= 1e-9 * p2) return l;  // after a quadratic step: l is the root
      break;                            // slow (multiple root): rounding limits l
    }
    const double step = -f / df;
    l += step;
    if (step <= 1e-17 * p2) return l;
    last = step;
  }
  double lam[3];
  sym3_eigenvalues(C, lam);
  return lam[0];
}

// One registration pair of a batch: where its points, padded records,
// partial sums and combine blocks live in the concatenated buffers.
struct BatchPair {
  int64_t x0, n;     // reference points [x0, x0 + n) of the concatenated reference cloud
  int64_t y0, m;     // template points [y0, y0 + m)
  int64_t xtile0;    // first force tile of this pair's reference records
  int64_t ybase;     // first padded template slot
  int64_t pbase;     // first per-chunk partial slot
  int64_t mpad;      // padded template slots (multiple of 256)
  int ntiles;        // reference tiles of FORCE_TJ points
  int chunks;        // reference chunks (one partial per chunk and template point)
  int cblk0, ncblk;  // combine blocks [cblk0, cblk0 + ncblk) of 256 template slots
  int shape4;        // mixed batched pass: 1 if this pair's force items take 4 template points x 128 threads
                     // (512-point blocks, running sums in shared memory), 0 for 2 points x 128 threads
};

// Uniform grid of the exact grid kNN: origin, cell edge, cells per axis.
struct GridSpec {
  double o[3];
  double h, inv_h;
  int g[3];
};

// ---- launchers (defined in the .cu files) --------------------------------
struct Launch {
  cudaStream_t stream;
  int64_t* counter;  // incremented once per kernel launch
};

cudaError_t launch_pack(Launch L, const float* xyz, int64_t n, float4* out, int* err);
cudaError_t launch_knn(Launch L, const float4* P, int n, int k, int32_t* out);
cudaError_t launch_curvature(Launch L, const float4* P, const int32_t* nbr, int n, int k,
                             double* a64, float* a32);
// mean + scatter of a cloud: writes mean[3], scatter[9], lmax of scatter/n
cudaError_t launch_cloud_stats(Launch L, const float4* P, int n, double* part, double* mean,
                               double* scatter, double* lmax);
// sigma = population std of a64 (1 if below 1e-12), or `sigma_user` if > 0
cudaError_t launch_sigma(Launch L, const double* a64, int n, double sigma_user, double* part,
                         double* sigma_out, double* asum_out);
cudaError_t launch_knn_multi(Launch L, const float4* P, const int64_t* off_dev, const int2* table_dev,
                             int nblocks, int k, int32_t* out);
cudaError_t launch_records_multi(Launch L, const float4* X4, const double* aX64, const float4* Y4,
                                 const double* aY64, const BatchPair* pairs, int npairs, int g_mode,
                                 const DevStats* stats, float4* Xr, float2* XA, float4* Y0r);
cudaError_t launch_stats_multi(Launch L, const float4* X4, const float4* Y4, const double* aX64,
                               const BatchPair* pairs, int npairs, double sigma_user, DevStats* out);
GridSpec make_grid_spec(const float* bbox6, int64_t n);
int64_t grid_cells(const GridSpec& gs);
cudaError_t launch_bbox(Launch L, const float4* P, int n, float* part, float* out6);
cudaError_t launch_knn_grid(Launch L, const float4* P, int n, int k, const GridSpec& gs, int* cell_of, int* count,
                            int* start, int* cursor, int* block_tot, float4* sorted, int* sorted_idx,
                            int32_t* out);
cudaError_t launch_nearest(Launch L, const float4* P, int n, const float* q3, int nq, int32_t* idx_out,
                           float* key_out);
cudaError_t launch_grid_build(Launch L, const float4* P, int n, const GridSpec& gs, int* cell_of, int* count,
                              int* start, int* cursor, int* block_tot, float4* sorted, int* sorted_idx);
constexpr int NEAREST_COARSE = 4;  // fine cells per coarse cell side in the two-level nearest search
GridSpec coarse_grid_spec(const GridSpec& gs);
cudaError_t launch_nearest_grid2(Launch L, const float4* sorted, const int* sorted_idx, const int* start,
                                 const GridSpec& gs, const float4* csorted, const int* csorted_idx,
                                 const int* cstart, const GridSpec& gc, const float* q3, int nq, int32_t* idx_out,
                                 float* key_out);
cudaError_t launch_nearest_grid(Launch L, const float4* sorted, const int* sorted_idx, const int* start,
                                const GridSpec& gs, const float* q3, int nq, int32_t* idx_out, float* key_out);
cudaError_t launch_threshold(Launch L, const float* key, int nq, float thr2, uint8_t* mask, float* dist);
cudaError_t launch_scale_double(Launch L, double* v, double f);
cudaError_t launch_radius_curvature(Launch L, const float4* P, int n, const double* e_dev, double scale2,
                                    double* a64, float* a32, int* count_out);
cudaError_t launch_check_curvature(Launch L, const double* a64, int n, float* a32, int* err);
cudaError_t launch_records(Launch L, const float4* X4, const double* aX64, int n, int npad,
                           const float4* Y4, const double* aY64, int m, int mpad, int g_mode,
                           const DevStats* stats, float4* Xr, float2* XA, float4* Y0r);

// Reference points per shared-memory tile of the force kernel; npad is a
// multiple of it.
constexpr int FORCE_TJ = 256;

struct ForcePlan {
  int P;          // template points per thread
  int tpb;        // threads per block
  int pmode;      // 1: p == 1, 2: p == 2, 3: p == 3, 0: general p, 4: p == 2 through rsqrt
  int tile_j;     // reference points per shared-memory tile
  int splits;     // reference-range splits (grid.y)
  int tiles_per_split;
  int iblocks;    // grid.x
  int occ;        // 0: >= 2 resident blocks per SM; 1: more (3 for 256 threads and P <= 2, 4 for 128 threads);
                  // 2: running sums in shared memory, 2 record tiles per stage (P = 4 x 128, P = 2 x 256)
  int ex2poly;    // p = 2, occ 2 only: number of template points per thread (0..2) whose second packed pair
                  // update of each 4-point step evaluates 2^-e on the FP32 pipe instead of the special-function
                  // unit (a fraction ex2poly / (2 P) of the pairs)
  int half;       // 1: each reference split is half a tile (splits = 2 ntiles; 1 point x 128 threads, problems
                  // whose one-tile grid fills less than half a wave)
};

// Overrides of the force plan (0: automatic), set by the autotuner.
struct ForceTuning {
  int P = 0;       // template points per thread: 1, 2 or 4
  int tpb = 0;     // threads per block: 128 or 256
  int splits = 0;  // reference splits
  int occ = -1;    // -1 automatic; 0 default; 1 the higher-occupancy variant (tighter register budget);
                   // 2 shared-memory sums
  int rsq = 0;     // p = 2 distance factor: 0 / 2 sqrt, 1 d^2 * rsqrt(d^2)
  int ex2poly = 0; // see ForcePlan::ex2poly
};

// blocks_per_sm > 0 replaces the device's occupancy query (host-only planning)
ForcePlan plan_force(int64_t m, int64_t npad, double p, int num_sms, const ForceTuning& tune = ForceTuning(),
                     int blocks_per_sm = 0);
int64_t force_mpad(int64_t m, const ForcePlan& fp);
// Record tiles a force block of this plan stages at a time (a split length
// that is not a multiple of this computes a zero-weight padded tile).
inline int force_stage_tiles(const ForcePlan& fp) { return fp.occ == 2 ? 2 : 1; }

cudaError_t launch_force(Launch L, const ForcePlan& fp, const float4* Xr, const float2* XA,
                         int ntiles, const float4* Y0r, int mpad, const DevPose* pose,
                         float qexp, float4* partial);
int combine_blocks(int64_t mpad);
cudaError_t launch_combine(Launch L, const float4* partial, int S, int mpad, int m,
                           const float4* Y0r, const float* aY32, int g_mode,
                           const DevPose* pose, float4* f4out, double* blockpart);
cudaError_t launch_pose_init(Launch L, DevPose* pose, const DevStats* stats, int E);
constexpr int FUSED_MAX_SLOTS = 2048;  // templates up to this many padded slots: combine_finalize_kernel
cudaError_t launch_combine_finalize(Launch L, const float4* partial, int S, int mpad, int m, const float4* Y0r,
                                    const float* aY32, int g_mode, DevPose* pose, const DevStats* stats,
                                    StepParams sp, int* err);
cudaError_t launch_finalize(Launch L, const double* blockpart, int nblocks, DevPose* pose,
                            const DevStats* stats, StepParams sp, int* err);
cudaError_t launch_apply(Launch L, const float4* Y4, int m, const DevPose* pose, float* out);
cudaError_t launch_pose_refresh(Launch L, DevPose* pose, const DevStats* stats);

int moments_splits(int ntiles, int num_sms, int64_t mpad);
cudaError_t launch_moments(Launch L, const float4* Xr, const float2* XA, int ntiles, const float4* Y0r, int mpad,
                           int m, int S, double* mpart, double* mom);
cudaError_t launch_combine_moments(Launch L, const double* mom, int m, int mpad, const float4* Y0r,
                                   const double* aY64, int g_mode, const DevPose* pose, float4* f4out,
                                   double* blockpart);
cudaError_t launch_force_batch(Launch L, int pmode, int P, int nitems, const int4* items, const BatchPair* pairs,
                               const float4* Xr, const float2* XA, const float4* Y0r, const DevPose* poses,
                               float qexp, float4* partial, int chunk_tiles, int grid, int* next);
// Resident blocks of the persistent batched force kernel (its `grid`).
cudaError_t force_batch_slots(int pmode, int P, int* slots);
// Threads per block of the batched force kernel with P template points per thread.
int batch_block_threads(int P);
bool batch_pair_shape4(int64_t m);
cudaError_t launch_combine_batch(Launch L, int nblocks, const int* cpair, const BatchPair* pairs,
                                 const float4* partial, const float4* Y0r, const float* aY32, int g_mode,
                                 const DevPose* poses, double* blockpart);
cudaError_t launch_finalize_multi(Launch L, const double* blockpart, const BatchPair* pairs, int npairs,
                                  DevPose* poses, const DevStats* stats, StepParams sp, int* err);
cudaError_t launch_pose_init_multi(Launch L, DevPose* poses, const DevStats* stats, int npairs, int E);
cudaError_t launch_force_vjp(Launch L, const float4* Xr, const float2* XA, int ntiles, const float4* Y0r,
                             const double* aY64, int g_mode, int m, const DevPose* ps, double p, const float* v,
                             float* grad);
// Stored pair terms: W is M rows of npad floats (npad = the padded reference
// length of the records, a multiple of 256).
cudaError_t launch_store_pairs(Launch L, const float2* XA, const float4* Xr, int npad, const float4* Y0r,
                               const double* aY64, int g_mode, int m, const DevPose* ps, float qexp, float* Wst,
                               double* Upart, double* Uout);
cudaError_t launch_stored_rows(Launch L, const float* Wst, int npad, int m, const float4* Xr, float4* partial);
int store_pairs_columns(int npad);   // grid columns of the store pass
int store_pairs_row_blocks(int m);   // grid rows of the store pass
cudaError_t launch_pose_from7(Launch L, const double* pose7_dev, DevPose* ps, const DevStats* st);
cudaError_t launch_adjoint_combine(Launch L, const float4* partial, int S, int mpad, int m, const float4* Y0r,
                                   const double* aY64, int g_mode, const DevPose* ps, float* grad_xyz,
                                   double* blockpart);
cudaError_t launch_column_sum13(Launch L, const double* part, int nb, double* out);
cudaError_t launch_adjoint_finish(Launch L, const double* tot, const double* pose7_dev, const DevPose* ps,
                                  double* grad7);

}  // namespace scgr
