// Shape-weighted potential and its adjoint (the differentiation form).
//
// U = sum_i sum_j g(s_ij) d_ij^(p+1) / (p+1) is the potential whose negative
// gradient with respect to Y_i is the force of Eq. 5 (descriptors fixed).
// With Y = s Y0 R(omega) + t (row vectors, R = exp([omega]_x)^T) the pose
// gradient follows from G_i = dU/dY_i = -f_i:
//   dU/dt = sum_i G_i,   dU/ds = sum_i G_i . (Y0_i R),
//   dU/dR = s sum_i Y0_i^T G_i,   dU/dY0_i = s G_i R^T,
// and for the axis-angle the SO(3) right Jacobian J_r: perturbing
// R_col(omega + delta) = R_col(omega) exp([J_r(omega) delta]_x) gives
// dU/domega = J_r(omega)^T w, where w is the axial vector of the skew part of
// B = (dU/dR) R_col (w_c = sum_ab eps_abc B_ab).
//
// The forward pass is the force kernel with the distance exponent raised by
// two (it accumulates sum_j g d^(p+1)); the adjoint pass re-runs the force
// kernel at the same pose (tile recomputation: no N x M storage) and reduces
// the chain-rule terms in float64 in a fixed order.
#include <cmath>

#include "common.cuh"

namespace scgr {

// Template point in the frame centred on the reference mean (identical
// arithmetic to the force kernel's).
__device__ __forceinline__ void tpoint(const float4 y0, const float* A, const float* b, float& yx,
                                       float& yy, float& yz) {
  yx = fmaf(y0.z, A[6], fmaf(y0.y, A[3], fmaf(y0.x, A[0], b[0])));
  yy = fmaf(y0.z, A[7], fmaf(y0.y, A[4], fmaf(y0.x, A[1], b[1])));
  yz = fmaf(y0.z, A[8], fmaf(y0.y, A[5], fmaf(y0.x, A[2], b[2])));
}

// Row-vector rotation R = exp([w]_x)^T by the Rodrigues formula.
__device__ void rotation_from_axis_angle(const double* w, double* R) {
  const double th2 = w[0] * w[0] + w[1] * w[1] + w[2] * w[2];
  double a, bq;  // exp([w]x) = I + a K + bq K^2
  if (th2 < 1e-16) {
    a = 1.0 - th2 / 6.0;
    bq = 0.5 - th2 / 24.0;
  } else {
    const double th = sqrt(th2);
    a = sin(th) / th;
    bq = (1.0 - cos(th)) / th2;
  }
  const double K[9] = {0.0, -w[2], w[1], w[2], 0.0, -w[0], -w[1], w[0], 0.0};
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c) {
      double k2 = 0.0;
      for (int q = 0; q < 3; ++q) k2 += K[r * 3 + q] * K[q * 3 + c];
      const double rc = (r == c ? 1.0 : 0.0) + a * K[r * 3 + c] + bq * k2;
      R[c * 3 + r] = rc;  // transpose: row-vector convention
    }
}

__global__ void pose_from7_kernel(const double* __restrict__ pose7, DevPose* ps, const DevStats* st) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  rotation_from_axis_angle(pose7, ps->R);
  for (int c = 0; c < 3; ++c) ps->t[c] = pose7[3 + c];
  ps->s = pose7[6];
  for (int q = 0; q < 9; ++q) ps->A[q] = (float)(ps->s * ps->R[q]);
  for (int c = 0; c < 3; ++c) {
    ps->b[c] = (float)(ps->t[c] - st->xbar[c]);
    const double yb = ps->s * (st->ybar0[0] * ps->R[c] + st->ybar0[1] * ps->R[3 + c] +
                               st->ybar0[2] * ps->R[6 + c]) + ps->t[c];
    set_ybs(ps, c, yb - st->xbar[c]);
  }
  ps->it = 0;
  ps->E = 1;
  ps->degenerate = 0;
}

// Per point: G_i = -f_i from the split partials; the template-coordinate
// gradient s G_i R^T; per-block chain-rule sums (sum G, sum G.(Y0 R),
// sum Y0^T G).
__global__ void __launch_bounds__(RED_THREADS)
    adjoint_combine_kernel(const float4* __restrict__ partial, int S, int mpad, int m,
                           const float4* __restrict__ Y0r, const double* __restrict__ aY64,
                           int g_mode, const DevPose* __restrict__ ps, float* __restrict__ grad_xyz,
                           double* __restrict__ blockpart) {
  __shared__ double sh[13][RED_THREADS];
  const int i = blockIdx.x * RED_THREADS + threadIdx.x;
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
    for (int q = 0; q < 9; ++q) A[q] = ps->A[q];
#pragma unroll
    for (int q = 0; q < 3; ++q) b[q] = ps->b[q];
    const float4 y0 = Y0r[i];
    float yx, yy, yz;
    tpoint(y0, A, b, yx, yy, yz);
    const double ay = g_mode == 1 ? aY64[i] : 1.0;
    // G = dU/dY = -f = aY (Y' sum w - sum w X')
    const double G[3] = {ay * ((double)yx * W - Sx), ay * ((double)yy * W - Sy), ay * ((double)yz * W - Sz)};
    const double Y0d[3] = {(double)y0.x, (double)y0.y, (double)y0.z};
    double y0R[3];
    for (int c = 0; c < 3; ++c)
      y0R[c] = Y0d[0] * ps->R[c] + Y0d[1] * ps->R[3 + c] + Y0d[2] * ps->R[6 + c];
    v[0] = G[0];
    v[1] = G[1];
    v[2] = G[2];
    v[3] = G[0] * y0R[0] + G[1] * y0R[1] + G[2] * y0R[2];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int bb = 0; bb < 3; ++bb) v[4 + 3 * a + bb] = Y0d[a] * G[bb];
    if (grad_xyz) {
      for (int a = 0; a < 3; ++a) {
        const double gr = ps->s * (G[0] * ps->R[a * 3] + G[1] * ps->R[a * 3 + 1] + G[2] * ps->R[a * 3 + 2]);
        grad_xyz[(size_t)i * 3 + a] = (float)gr;
      }
    }
  }
  block_sum<13>(v, sh);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int q = 0; q < 13; ++q) blockpart[(size_t)blockIdx.x * 13 + q] = v[q];
  }
}

// One block: fixed-order column sums of [nb][13] partials.
__global__ void __launch_bounds__(RED_THREADS) column_sum13_kernel(const double* __restrict__ part, int nb,
                                                                   double* __restrict__ out) {
  __shared__ double sh[13][RED_THREADS];
  double v[13];
#pragma unroll
  for (int q = 0; q < 13; ++q) v[q] = 0.0;
  for (int b = threadIdx.x; b < nb; b += RED_THREADS) {
#pragma unroll
    for (int q = 0; q < 13; ++q) v[q] += part[(size_t)b * 13 + q];
  }
  block_sum<13>(v, sh);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int q = 0; q < 13; ++q) out[q] = v[q];
  }
}

// grad7 = (dU/domega, dU/dt, dU/ds) from the chain-rule sums.
__global__ void adjoint_finish_kernel(const double* __restrict__ tot, const double* __restrict__ pose7,
                                      const DevPose* __restrict__ ps, double* __restrict__ grad7) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const double s = ps->s;
  double M[9];  // dU/dR
  for (int q = 0; q < 9; ++q) M[q] = s * tot[4 + q];
  // B = M R_col, R_col = R^T
  double B[9];
  for (int a = 0; a < 3; ++a)
    for (int c = 0; c < 3; ++c) {
      double acc = 0.0;
      for (int q = 0; q < 3; ++q) acc += M[a * 3 + q] * ps->R[c * 3 + q];
      B[a * 3 + c] = acc;
    }
  const double w[3] = {B[5] - B[7], B[6] - B[2], B[1] - B[3]};
  const double* om = pose7;
  const double th2 = om[0] * om[0] + om[1] * om[1] + om[2] * om[2];
  double c1, c2;  // J_r = I - c1 K + c2 K^2
  if (th2 < 1e-12) {
    c1 = 0.5 - th2 / 24.0;
    c2 = 1.0 / 6.0 - th2 / 120.0;
  } else {
    const double th = sqrt(th2);
    c1 = (1.0 - cos(th)) / th2;
    c2 = (th - sin(th)) / (th2 * th);
  }
  const double K[9] = {0.0, -om[2], om[1], om[2], 0.0, -om[0], -om[1], om[0], 0.0};
  double J[9];
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c) {
      double k2 = 0.0;
      for (int q = 0; q < 3; ++q) k2 += K[r * 3 + q] * K[q * 3 + c];
      J[r * 3 + c] = (r == c ? 1.0 : 0.0) - c1 * K[r * 3 + c] + c2 * k2;
    }
  for (int k = 0; k < 3; ++k) grad7[k] = J[0 * 3 + k] * w[0] + J[1 * 3 + k] * w[1] + J[2 * 3 + k] * w[2];
  for (int c = 0; c < 3; ++c) grad7[3 + c] = tot[c];
  grad7[6] = tot[3];
}

// ---- vector-Jacobian product of the force field ---------------------------
// f_i depends on Y_i only (X fixed, descriptors fixed), so dF/dY is block
// diagonal with J_ii = -aY sum_j w_ij [I + (p - 1) r r^T / d^2], r = Y_i - X_j,
// w_ij = g d^(p-1).  grad_i = J_ii v_i (J_ii is symmetric).  One thread per
// template point; reference tiles of the force records are recomputed.
constexpr int VJP_TPB = 128;
constexpr int VJP_TILE = FORCE_TJ;

__global__ void __launch_bounds__(VJP_TPB)
    force_vjp_kernel(const float* __restrict__ Xr, const float* __restrict__ XA, int ntiles,
                     const float4* __restrict__ Y0r, const double* __restrict__ aY64, int g_mode, int m,
                     const DevPose* __restrict__ ps, double pm1, const float* __restrict__ v,
                     float* __restrict__ grad) {
  __shared__ float sT[6][VJP_TILE];
  const int i = blockIdx.x * VJP_TPB + threadIdx.x;
  float A[9], b[3];
#pragma unroll
  for (int q = 0; q < 9; ++q) A[q] = ps->A[q];
#pragma unroll
  for (int q = 0; q < 3; ++q) b[q] = ps->b[q];
  const float4 y0 = Y0r[i < m ? i : m - 1];
  float yx, yy, yz;
  tpoint(y0, A, b, yx, yy, yz);
  const float ah = y0.w;
  const float q = (float)(0.5 * pm1);           // d^(p-1) = (d^2)^q
  double Ws = 0.0, B[6] = {0, 0, 0, 0, 0, 0};   // sum w, sum w (p-1) r r^T / d^2
  for (int t = 0; t < ntiles; ++t) {
    __syncthreads();
    for (int u = threadIdx.x; u < 4 * VJP_TILE; u += VJP_TPB) (&sT[0][0])[u] = Xr[(size_t)t * 4 * VJP_TILE + u];
    for (int u = threadIdx.x; u < 2 * VJP_TILE; u += VJP_TPB) (&sT[4][0])[u] = XA[(size_t)t * 2 * VJP_TILE + u];
    __syncthreads();
    float ws = 0.f, bb[6] = {0, 0, 0, 0, 0, 0};
    for (int j = 0; j < VJP_TILE; ++j) {
      const float rx = yx - sT[0][j], ry = yy - sT[1][j], rz = yz - sT[2][j];
      const float d2 = fmaf(rz, rz, fmaf(ry, ry, rx * rx));
      const float uu = sT[4][j] - ah;
      const float ep = fmaf(uu, uu, sT[5][j]);  // the weight is 2^-ep d^(p-1)
      const float w = d2 > 0.f ? exp2f(fmaf(q, log2f(d2), -ep)) : (q == 0.f ? exp2f(-ep) : 0.f);
      const float c = d2 > 0.f ? (float)pm1 * w / d2 : 0.f;
      ws += w;
      bb[0] = fmaf(c * rx, rx, bb[0]); bb[1] = fmaf(c * rx, ry, bb[1]); bb[2] = fmaf(c * rx, rz, bb[2]);
      bb[3] = fmaf(c * ry, ry, bb[3]); bb[4] = fmaf(c * ry, rz, bb[4]); bb[5] = fmaf(c * rz, rz, bb[5]);
    }
    Ws += ws;
    for (int u = 0; u < 6; ++u) B[u] += bb[u];
  }
  if (i >= m) return;
  const double ay = g_mode == 1 ? aY64[i] : 1.0;
  const double vx = v[3 * (size_t)i], vy = v[3 * (size_t)i + 1], vz = v[3 * (size_t)i + 2];
  const double gx = -ay * (Ws * vx + B[0] * vx + B[1] * vy + B[2] * vz);
  const double gy = -ay * (Ws * vy + B[1] * vx + B[3] * vy + B[4] * vz);
  const double gz = -ay * (Ws * vz + B[2] * vx + B[4] * vy + B[5] * vz);
  grad[3 * (size_t)i] = (float)gx;
  grad[3 * (size_t)i + 1] = (float)gy;
  grad[3 * (size_t)i + 2] = (float)gz;
}

cudaError_t launch_force_vjp(Launch L, const float4* Xr, const float2* XA, int ntiles, const float4* Y0r,
                             const double* aY64, int g_mode, int m, const DevPose* ps, double p, const float* v,
                             float* grad) {
  if (m <= 0) return cudaSuccess;
  force_vjp_kernel<<<(m + VJP_TPB - 1) / VJP_TPB, VJP_TPB, 0, L.stream>>>(
      reinterpret_cast<const float*>(Xr), reinterpret_cast<const float*>(XA), ntiles, Y0r, aY64, g_mode, m, ps,
      p - 1.0, v, grad);
  if (L.counter) ++*L.counter;
  return cudaGetLastError();
}

// ---- stored pair terms (comparison variant of the adjoint) -----------------
// Forward: every pair weight w_ij = g d^(p-1) is written to W[i][npad]
// (float32, M rows of the padded reference length; padding records carry
// weight 0) and the potential U = sum aY w d^2 / (p + 1) is summed per block.
// Backward: a block streams ST_RROWS rows back from HBM and forms the same
// per-point sums (sum w, sum w X') that the force kernel accumulates, so the
// adjoint reduction is shared.  Both passes move 16 bytes per thread access:
// a thread owns four consecutive reference points.
constexpr int ST_TPB = 256;
constexpr int ST_JB = 4 * ST_TPB;  // reference points per block column (npad is a multiple of it or of 256)

// Block (ST_ROWS template points x ST_JB reference points): the records are
// read once, each thread walks the block's template points and writes each
// row segment as one float4.
constexpr int ST_ROWS = 64;

__device__ __forceinline__ float st_ex2(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float st_lg2(float x) {
  float y;
  asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// w = 2^-(u^2 - L) d^(p-1) with d^(p-1) = 2^(qexp log2 d^2), qexp = (p-1)/2.
__device__ __forceinline__ float st_weight(float d2, float ep, float qexp) {
  if (qexp == 0.f) return st_ex2(-ep);
  return st_ex2(fmaf(qexp, st_lg2(d2), -ep));  // d2 = 0: lg2 = -inf, weight 0
}

__global__ void __launch_bounds__(ST_TPB)
    store_pairs_kernel(const float* __restrict__ Xr, const float* __restrict__ XA, int npad, int m,
                       const float4* __restrict__ Y0r, const double* __restrict__ aY64, int g_mode,
                       const DevPose* __restrict__ ps, float qexp, float* __restrict__ Wst,
                       double* __restrict__ Upart) {
  __shared__ double sh[1][RED_THREADS];
  const int j0 = blockIdx.y * ST_JB + threadIdx.x * 4;
  const int i0 = blockIdx.x * ST_ROWS;
  float A[9], b[3];
#pragma unroll
  for (int q = 0; q < 9; ++q) A[q] = ps->A[q];
#pragma unroll
  for (int q = 0; q < 3; ++q) b[q] = ps->b[q];
  float4 x4 = make_float4(0.f, 0.f, 0.f, 0.f), y4 = x4, z4 = x4, a4 = x4;
  float4 l4 = make_float4(INFINITY, INFINITY, INFINITY, INFINITY);
  const bool live = j0 < npad;
  if (live) {
    const size_t t = (size_t)(j0 / FORCE_TJ), r = (size_t)(j0 % FORCE_TJ);
    const float* xr = Xr + t * 4 * FORCE_TJ + r;
    const float* xa = XA + t * 2 * FORCE_TJ + r;
    x4 = *reinterpret_cast<const float4*>(xr);
    y4 = *reinterpret_cast<const float4*>(xr + FORCE_TJ);
    z4 = *reinterpret_cast<const float4*>(xr + 2 * FORCE_TJ);
    a4 = *reinterpret_cast<const float4*>(xa);
    l4 = *reinterpret_cast<const float4*>(xa + FORCE_TJ);
  }
  const float xs[4] = {x4.x, x4.y, x4.z, x4.w}, ys[4] = {y4.x, y4.y, y4.z, y4.w};
  const float zs[4] = {z4.x, z4.y, z4.z, z4.w}, as[4] = {a4.x, a4.y, a4.z, a4.w};
  const float ls[4] = {l4.x, l4.y, l4.z, l4.w};
  // U terms are summed in FP32 over runs of 16 rows and the runs in FP64
  // (FP64 arithmetic per pair would cost more than the pair itself).
  double u[1] = {0.0};
  const int iend = min(m, i0 + ST_ROWS);
  for (int ib = i0; ib < iend; ib += 16) {
    float run = 0.f;
    const int ie = min(iend, ib + 16);
    for (int i = ib; i < ie; ++i) {
      const float4 y0 = Y0r[i];
      float yx, yy, yz;
      tpoint(y0, A, b, yx, yy, yz);
      const float ay = g_mode == 1 ? (float)aY64[i] : 1.f;
      float w[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const float rx = yx - xs[k], ry = yy - ys[k], rz = yz - zs[k];
        const float d2 = fmaf(rz, rz, fmaf(ry, ry, rx * rx));
        const float uu = as[k] - y0.w;
        w[k] = st_weight(d2, fmaf(uu, uu, ls[k]), qexp);
        run = fmaf(ay * w[k], d2, run);
      }
      if (live) *reinterpret_cast<float4*>(Wst + (size_t)i * npad + j0) = make_float4(w[0], w[1], w[2], w[3]);
    }
    u[0] += (double)run;
  }
  block_sum<1>(u, sh);
  if (threadIdx.x == 0) Upart[(size_t)blockIdx.x * gridDim.y + blockIdx.y] = u[0];
}

// Backward from the stored weights: a block owns ST_RROWS template rows and
// each thread four consecutive reference points per step, so every weight is
// read once as part of a float4 (all ST_RROWS loads of a step are issued
// before they are used) and each reference record once per block.  The last
// block re-reads row m-1 for its missing rows and discards those sums.
constexpr int ST_RROWS = 8;

__global__ void __launch_bounds__(ST_TPB, 2)
    stored_rows_kernel(const float* __restrict__ Wst, int npad, int m, const float* __restrict__ Xr,
                       float4* __restrict__ partial) {
  __shared__ double red[ST_TPB / 32][ST_RROWS * 4];
  const int r0 = blockIdx.x * ST_RROWS;
  const int nr = min(ST_RROWS, m - r0);
  const float* rows[ST_RROWS];
#pragma unroll
  for (int r = 0; r < ST_RROWS; ++r) rows[r] = Wst + (size_t)min(r0 + r, m - 1) * npad;
  float acc[ST_RROWS][4];
#pragma unroll
  for (int r = 0; r < ST_RROWS; ++r) acc[r][0] = acc[r][1] = acc[r][2] = acc[r][3] = 0.f;
  for (int j0 = threadIdx.x * 4; j0 < npad; j0 += ST_JB) {
    float4 w4[ST_RROWS];
#pragma unroll
    for (int r = 0; r < ST_RROWS; ++r) w4[r] = *reinterpret_cast<const float4*>(rows[r] + j0);
    const size_t t = (size_t)(j0 / FORCE_TJ), q = (size_t)(j0 % FORCE_TJ);
    const float* xr = Xr + t * 4 * FORCE_TJ + q;
    const float4 x = *reinterpret_cast<const float4*>(xr);
    const float4 y = *reinterpret_cast<const float4*>(xr + FORCE_TJ);
    const float4 z = *reinterpret_cast<const float4*>(xr + 2 * FORCE_TJ);
#pragma unroll
    for (int r = 0; r < ST_RROWS; ++r) {
      const float4 w = w4[r];
      acc[r][0] += (w.x + w.y) + (w.z + w.w);
      acc[r][1] = fmaf(w.w, x.w, fmaf(w.z, x.z, fmaf(w.y, x.y, fmaf(w.x, x.x, acc[r][1]))));
      acc[r][2] = fmaf(w.w, y.w, fmaf(w.z, y.z, fmaf(w.y, y.y, fmaf(w.x, y.x, acc[r][2]))));
      acc[r][3] = fmaf(w.w, z.w, fmaf(w.z, z.z, fmaf(w.y, z.y, fmaf(w.x, z.x, acc[r][3]))));
    }
  }
  // block reduction: FP32 warp shuffles, then the warps' sums in FP64
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int r = 0; r < ST_RROWS; ++r)
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      float v = acc[r][c];
      for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
      if (lane == 0) red[warp][r * 4 + c] = v;
    }
  __syncthreads();
  if (threadIdx.x < ST_RROWS * 4) {
    double v = 0.0;
    for (int w = 0; w < ST_TPB / 32; ++w) v += red[w][threadIdx.x];
    red[0][threadIdx.x] = v;
  }
  __syncthreads();
  if (threadIdx.x < nr)
    partial[r0 + threadIdx.x] = make_float4((float)red[0][threadIdx.x * 4], (float)red[0][threadIdx.x * 4 + 1],
                                            (float)red[0][threadIdx.x * 4 + 2], (float)red[0][threadIdx.x * 4 + 3]);
}

__global__ void __launch_bounds__(RED_THREADS) sum_rows_kernel(const double* __restrict__ part, int64_t count,
                                                               double* __restrict__ out) {
  __shared__ double sh[1][RED_THREADS];
  double v[1] = {0.0};
  for (int64_t q = threadIdx.x; q < count; q += RED_THREADS) v[0] += part[q];
  block_sum<1>(v, sh);
  if (threadIdx.x == 0) out[0] = v[0];
}

cudaError_t launch_store_pairs(Launch L, const float2* XA, const float4* Xr, int npad, const float4* Y0r,
                               const double* aY64, int g_mode, int m, const DevPose* ps, float qexp, float* Wst,
                               double* Upart, double* Uout) {
  const int nb = store_pairs_columns(npad);
  const int ib = (m + ST_ROWS - 1) / ST_ROWS;
  store_pairs_kernel<<<dim3(ib, nb), ST_TPB, 0, L.stream>>>(reinterpret_cast<const float*>(Xr),
                                                           reinterpret_cast<const float*>(XA), npad, m, Y0r, aY64,
                                                           g_mode, ps, qexp, Wst, Upart);
  sum_rows_kernel<<<1, RED_THREADS, 0, L.stream>>>(Upart, (int64_t)nb * ib, Uout);
  if (L.counter) *L.counter += 2;
  return cudaGetLastError();
}

int store_pairs_columns(int npad) { return (npad + ST_JB - 1) / ST_JB; }
int store_pairs_row_blocks(int m) { return (m + ST_ROWS - 1) / ST_ROWS; }

cudaError_t launch_stored_rows(Launch L, const float* Wst, int npad, int m, const float4* Xr, float4* partial) {
  stored_rows_kernel<<<(m + ST_RROWS - 1) / ST_RROWS, ST_TPB, 0, L.stream>>>(Wst, npad, m,
                                                                            reinterpret_cast<const float*>(Xr), partial);
  if (L.counter) ++*L.counter;
  return cudaGetLastError();
}

cudaError_t launch_pose_from7(Launch L, const double* pose7_dev, DevPose* ps, const DevStats* st) {
  pose_from7_kernel<<<1, 32, 0, L.stream>>>(pose7_dev, ps, st);
  if (L.counter) ++*L.counter;
  return cudaGetLastError();
}

cudaError_t launch_adjoint_combine(Launch L, const float4* partial, int S, int mpad, int m, const float4* Y0r,
                                   const double* aY64, int g_mode, const DevPose* ps, float* grad_xyz,
                                   double* blockpart) {
  adjoint_combine_kernel<<<(mpad + RED_THREADS - 1) / RED_THREADS, RED_THREADS, 0, L.stream>>>(
      partial, S, mpad, m, Y0r, aY64, g_mode, ps, grad_xyz, blockpart);
  if (L.counter) ++*L.counter;
  return cudaGetLastError();
}

cudaError_t launch_column_sum13(Launch L, const double* part, int nb, double* out) {
  column_sum13_kernel<<<1, RED_THREADS, 0, L.stream>>>(part, nb, out);
  if (L.counter) ++*L.counter;
  return cudaGetLastError();
}

cudaError_t launch_adjoint_finish(Launch L, const double* tot, const double* pose7_dev, const DevPose* ps,
                                  double* grad7) {
  adjoint_finish_kernel<<<1, 32, 0, L.stream>>>(tot, pose7_dev, ps, grad7);
  if (L.counter) ++*L.counter;
  return cudaGetLastError();
}

}  // namespace scgr
