// All-pairs shape-weighted force (Eq. 5 with Eq. 3, Eq. 10, Eq. 11) and its
// reduction to the total force, weight and torque moment (Eq. 5.5, Eq. 6).
//
// For template point Y_i (M of them) and reference point X_j (N of them):
//   w_ij = g(s_ij) d_ij^(p-1),   f_i = -sum_j w_ij (Y_i - X_j),
//   W_i  = sum_j w_ij.
// The kernel accumulates, per template point, sum_j w_ij and sum_j w_ij X_j;
// f_i = aY (sum_j w X_j - Y_i sum_j w) is formed afterwards in float64.
//
// Per pair (float32): d^2 = |X'|^2 + |Y'|^2 - 2 X'.Y' (one add, three FMAs),
// the similarity-and-aX factor 2^(L - (a_hat_X - a_hat_Y)^2) (one add, one
// FMA, one ex2), the distance factor (sqrt for p = 2, folded into the ex2
// exponent through lg2 for general p), and four accumulations.  ex2 and the
// distance MUFU op are the only special-function instructions.
//
// Layout of the work: grid.x covers template points (P per thread, TPB
// threads), grid.y splits the reference range so that the grid has many
// waves on 152 SMs.  Reference tiles of TJ points are staged in shared
// memory and read as broadcasts.  Each tile's sums are accumulated in plain
// float32 and then added to the running per-point sums with Kahan
// compensation; each split writes its per-point partial (float4) and the
// combine kernel adds the splits in a fixed order in float64, so results are
// deterministic.
#include <cmath>

#include "common.cuh"

namespace scgr {

__device__ __forceinline__ float ex2_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float lg2_approx(float x) {
  float y;
  asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float sqrt_approx(float x) {
  float y;
  asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// Template point in the frame centred on the reference mean: Y' = Y0 A + b.
// The force and combine kernels both call this, so they see identical bits.
__device__ __forceinline__ void template_point(const float4 y0, const float* A, const float* b,
                                               float& yx, float& yy, float& yz) {
  yx = fmaf(y0.z, A[6], fmaf(y0.y, A[3], fmaf(y0.x, A[0], b[0])));
  yy = fmaf(y0.z, A[7], fmaf(y0.y, A[4], fmaf(y0.x, A[1], b[1])));
  yz = fmaf(y0.z, A[8], fmaf(y0.y, A[5], fmaf(y0.x, A[2], b[2])));
}

__device__ __forceinline__ void kahan_add(float& s, float& c, float x) {
  const float y = x - c;
  const float t = s + y;
  c = (t - s) - y;
  s = t;
}

template <int P, int PM, int TPB, int TJ, int MINB>
__global__ void __launch_bounds__(TPB, MINB)
    force_tile_kernel(const float4* __restrict__ Xr, const float2* __restrict__ XA, int ntiles,
                      int tiles_per_split, const float4* __restrict__ Y0r, int mpad,
                      const DevPose* __restrict__ pose, float qexp, float4* __restrict__ partial) {
  __shared__ float4 sX[TJ];
  __shared__ float2 sA[TJ];
  const int tid = threadIdx.x;
  const int ibase = blockIdx.x * (TPB * P);
  const int split = blockIdx.y;

  float A[9], b[3];
#pragma unroll
  for (int q = 0; q < 9; ++q) A[q] = pose->A[q];
#pragma unroll
  for (int q = 0; q < 3; ++q) b[q] = pose->b[q];

  float m2x[P], m2y[P], m2z[P], nY[P], ah[P];
#pragma unroll
  for (int q = 0; q < P; ++q) {
    const float4 y0 = Y0r[ibase + q * TPB + tid];
    float yx, yy, yz;
    template_point(y0, A, b, yx, yy, yz);
    m2x[q] = -2.f * yx;
    m2y[q] = -2.f * yy;
    m2z[q] = -2.f * yz;
    nY[q] = fmaf(yz, yz, fmaf(yy, yy, yx * yx));
    ah[q] = y0.w;
  }

  float hW[P], hx[P], hy[P], hz[P];  // running sums
  float cW[P], cx[P], cy[P], cz[P];  // Kahan compensations
#pragma unroll
  for (int q = 0; q < P; ++q) {
    hW[q] = hx[q] = hy[q] = hz[q] = 0.f;
    cW[q] = cx[q] = cy[q] = cz[q] = 0.f;
  }

  const int t0 = split * tiles_per_split;
  const int t1 = min(ntiles, t0 + tiles_per_split);
  for (int t = t0; t < t1; ++t) {
    __syncthreads();
#pragma unroll
    for (int u = tid; u < TJ; u += TPB) {
      sX[u] = Xr[(size_t)t * TJ + u];
      sA[u] = XA[(size_t)t * TJ + u];
    }
    __syncthreads();

    float aW[P], ax[P], ay[P], az[P];
#pragma unroll
    for (int q = 0; q < P; ++q) aW[q] = ax[q] = ay[q] = az[q] = 0.f;

#pragma unroll 2
    for (int jj = 0; jj < TJ; ++jj) {
      const float4 xr = sX[jj];
      const float2 xa = sA[jj];
#pragma unroll
      for (int q = 0; q < P; ++q) {
        float d2 = xr.w + nY[q];
        d2 = fmaf(xr.x, m2x[q], d2);
        d2 = fmaf(xr.y, m2y[q], d2);
        d2 = fmaf(xr.z, m2z[q], d2);
        const float u = xa.x - ah[q];
        const float e = fmaf(-u, u, xa.y);
        float w;
        if (PM == 1) {
          w = ex2_approx(e);
        } else if (PM == 2) {
          w = ex2_approx(e) * sqrt_approx(fabsf(d2));
        } else if (PM == 3) {
          w = ex2_approx(e) * fabsf(d2);
        } else {
          w = ex2_approx(fmaf(qexp, lg2_approx(fabsf(d2)), e));
        }
        aW[q] += w;
        ax[q] = fmaf(w, xr.x, ax[q]);
        ay[q] = fmaf(w, xr.y, ay[q]);
        az[q] = fmaf(w, xr.z, az[q]);
      }
    }
#pragma unroll
    for (int q = 0; q < P; ++q) {
      kahan_add(hW[q], cW[q], aW[q]);
      kahan_add(hx[q], cx[q], ax[q]);
      kahan_add(hy[q], cy[q], ay[q]);
      kahan_add(hz[q], cz[q], az[q]);
    }
  }

  float4* out = partial + (size_t)split * mpad + ibase + tid;
#pragma unroll
  for (int q = 0; q < P; ++q)
    out[q * TPB] = make_float4(hW[q] - cW[q], hx[q] - cx[q], hy[q] - cy[q], hz[q] - cz[q]);
}

// ---- planning --------------------------------------------------------------
constexpr int FORCE_TJ = 256;

ForcePlan plan_force(int64_t m, int64_t npad, double p, int num_sms) {
  ForcePlan fp;
  fp.pmode = (p == 1.0) ? 1 : (p == 2.0) ? 2 : (p == 3.0) ? 3 : 0;
  fp.tile_j = FORCE_TJ;
  fp.tpb = 256;
  // points per thread: the largest that still gives every SM work
  if (m >= (int64_t)num_sms * 2 * 256 * 4) fp.P = 4;
  else if (m >= (int64_t)num_sms * 256 * 2) fp.P = 2;
  else fp.P = 1;
  if (m < 4096) fp.tpb = 128;
  const int64_t per_block = (int64_t)fp.tpb * fp.P;
  fp.iblocks = (int)((m + per_block - 1) / per_block);
  const int ntiles = (int)(npad / FORCE_TJ);
  // aim for >= 16 waves of 2 resident blocks per SM, split the reference
  // range to get there, but keep >= 4 tiles per split
  const int64_t target = (int64_t)num_sms * 2 * 16;
  int64_t S = (target + fp.iblocks - 1) / fp.iblocks;
  int64_t Smax = ntiles / 4 > 0 ? ntiles / 4 : 1;
  if (S > Smax) S = Smax;
  if (S > 64) S = 64;
  if (S < 1) S = 1;
  fp.tiles_per_split = (int)((ntiles + S - 1) / S);
  fp.splits = (ntiles + fp.tiles_per_split - 1) / fp.tiles_per_split;
  return fp;
}

int64_t force_mpad(int64_t m, const ForcePlan& fp) {
  const int64_t per_block = (int64_t)fp.tpb * fp.P;
  int64_t mp = (m + per_block - 1) / per_block * per_block;
  // the combine kernel works in blocks of 256
  return (mp + 255) / 256 * 256;
}

template <int P, int PM, int TPB>
static void launch_force_t(cudaStream_t st, const ForcePlan& fp, const float4* Xr,
                           const float2* XA, int ntiles, const float4* Y0r, int mpad,
                           const DevPose* pose, float qexp, float4* partial) {
  dim3 grid(fp.iblocks, fp.splits);
  force_tile_kernel<P, PM, TPB, FORCE_TJ, 2><<<grid, TPB, 0, st>>>(
      Xr, XA, ntiles, fp.tiles_per_split, Y0r, mpad, pose, qexp, partial);
}

template <int PM>
static void launch_force_pm(cudaStream_t st, const ForcePlan& fp, const float4* Xr,
                            const float2* XA, int ntiles, const float4* Y0r, int mpad,
                            const DevPose* pose, float qexp, float4* partial) {
  if (fp.tpb == 256) {
    if (fp.P == 4) launch_force_t<4, PM, 256>(st, fp, Xr, XA, ntiles, Y0r, mpad, pose, qexp, partial);
    else if (fp.P == 2) launch_force_t<2, PM, 256>(st, fp, Xr, XA, ntiles, Y0r, mpad, pose, qexp, partial);
    else launch_force_t<1, PM, 256>(st, fp, Xr, XA, ntiles, Y0r, mpad, pose, qexp, partial);
  } else {
    launch_force_t<1, PM, 128>(st, fp, Xr, XA, ntiles, Y0r, mpad, pose, qexp, partial);
  }
}

cudaError_t launch_force(Launch L, const ForcePlan& fp, const float4* Xr, const float2* XA,
                         int ntiles, const float4* Y0r, int mpad, const DevPose* pose, float qexp,
                         float4* partial) {
  switch (fp.pmode) {
    case 1: launch_force_pm<1>(L.stream, fp, Xr, XA, ntiles, Y0r, mpad, pose, qexp, partial); break;
    case 2: launch_force_pm<2>(L.stream, fp, Xr, XA, ntiles, Y0r, mpad, pose, qexp, partial); break;
    case 3: launch_force_pm<3>(L.stream, fp, Xr, XA, ntiles, Y0r, mpad, pose, qexp, partial); break;
    default: launch_force_pm<0>(L.stream, fp, Xr, XA, ntiles, Y0r, mpad, pose, qexp, partial); break;
  }
  if (L.counter) ++*L.counter;
  return cudaGetLastError();
}

// ---- combine: splits -> per-point force -> per-block (F, W, T) -------------
constexpr int CMB_TPB = RED_THREADS;

__global__ void __launch_bounds__(CMB_TPB)
    combine_kernel(const float4* __restrict__ partial, int S, int mpad, int m,
                   const float4* __restrict__ Y0r, const double* __restrict__ aY64, int g_mode,
                   const DevPose* __restrict__ pose, float4* __restrict__ f4out,
                   double* __restrict__ blockpart) {
  __shared__ double sh[13][RED_THREADS];
  const int i = blockIdx.x * CMB_TPB + threadIdx.x;
  double v[13];
#pragma unroll
  for (int q = 0; q < 13; ++q) v[q] = 0.0;
  if (i < m) {
    double W = 0, Sx = 0, Sy = 0, Sz = 0;
    for (int s = 0; s < S; ++s) {
      const float4 pp = partial[(size_t)s * mpad + i];
      W += pp.x;
      Sx += pp.y;
      Sy += pp.z;
      Sz += pp.w;
    }
    float A[9], b[3];
#pragma unroll
    for (int q = 0; q < 9; ++q) A[q] = pose->A[q];
#pragma unroll
    for (int q = 0; q < 3; ++q) b[q] = pose->b[q];
    float yx, yy, yz;
    template_point(Y0r[i], A, b, yx, yy, yz);
    const double ay = g_mode == 1 ? aY64[i] : 1.0;
    const double f[3] = {ay * (Sx - (double)yx * W), ay * (Sy - (double)yy * W),
                         ay * (Sz - (double)yz * W)};
    const double Wi = ay * W;
    const double c[3] = {(double)yx - pose->ybs[0], (double)yy - pose->ybs[1],
                         (double)yz - pose->ybs[2]};
    v[0] = f[0];
    v[1] = f[1];
    v[2] = f[2];
    v[3] = Wi;
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int bb = 0; bb < 3; ++bb) v[4 + 3 * a + bb] = f[a] * c[bb];
    if (f4out) f4out[i] = make_float4((float)f[0], (float)f[1], (float)f[2], (float)Wi);
  }
  block_sum<13>(v, sh);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int q = 0; q < 13; ++q) blockpart[(size_t)blockIdx.x * 13 + q] = v[q];
  }
}

int combine_blocks(int64_t mpad) { return (int)((mpad + CMB_TPB - 1) / CMB_TPB); }

cudaError_t launch_combine(Launch L, const float4* partial, int S, int mpad, int m,
                           const float4* Y0r, const double* aY64, int g_mode, const DevPose* pose,
                           float4* f4out, double* blockpart) {
  combine_kernel<<<combine_blocks(mpad), CMB_TPB, 0, L.stream>>>(partial, S, mpad, m, Y0r, aY64,
                                                                 g_mode, pose, f4out, blockpart);
  if (L.counter) ++*L.counter;
  return cudaGetLastError();
}

}  // namespace scgr
