// Pose update in float64 (Eq. 5.5, Eq. 6, Eq. 8, Eq. 9, Eq. 12): one block
// reduces the per-block (F, W, T) partials in a fixed order, then one warp
// forms the step, the Kabsch rotation (the polar factor of C^ by Newton's
// iteration in float32 with float64 corrections, else in float64, or a
// one-sided Jacobi SVD in the reflection and near-singular cases), the
// scale, the composed pose and its re-orthonormalisation.  The pose never
// leaves the device, so a run of iterations is a plain sequence of launches.
#include <cmath>

#include "common.cuh"
#include "pointsum.cuh"

namespace scgr {

// A = U diag(S) V^T for a 3x3 A (row-major), S descending, U and V proper
// or improper orthogonal; one-sided Jacobi (Hestenes) rotations on columns.
__device__ void svd3(const double* Ain, double* U, double* S, double* V) {
  double a[3][3], v[3][3];
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c) {
      a[r][c] = Ain[r * 3 + c];
      v[r][c] = (r == c) ? 1.0 : 0.0;
    }
  for (int sweep = 0; sweep < 60; ++sweep) {
    double worst = 0.0;
    for (int pq = 0; pq < 3; ++pq) {
      const int p = pq == 2 ? 1 : 0;
      const int q = pq == 0 ? 1 : 2;
      double al = 0, be = 0, ga = 0;
      for (int k = 0; k < 3; ++k) {
        al += a[k][p] * a[k][p];
        be += a[k][q] * a[k][q];
        ga += a[k][p] * a[k][q];
      }
      if (ga == 0.0) continue;
      const double rel = fabs(ga) / sqrt(al * be);
      if (rel > worst) worst = rel;
      if (rel < 1e-16) continue;
      const double zeta = (be - al) / (2.0 * ga);
      double t;
      if (fabs(zeta) > 1e150) t = 0.5 / zeta;
      else t = (zeta >= 0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
      const double c = 1.0 / sqrt(1.0 + t * t);
      const double s = c * t;
      for (int k = 0; k < 3; ++k) {
        const double ap = a[k][p], aq = a[k][q];
        a[k][p] = c * ap - s * aq;
        a[k][q] = s * ap + c * aq;
        const double vp = v[k][p], vq = v[k][q];
        v[k][p] = c * vp - s * vq;
        v[k][q] = s * vp + c * vq;
      }
    }
    if (worst < 1e-15) break;
  }
  double sg[3];
  for (int p = 0; p < 3; ++p) sg[p] = sqrt(a[0][p] * a[0][p] + a[1][p] * a[1][p] + a[2][p] * a[2][p]);
  int o[3] = {0, 1, 2};
  for (int x = 0; x < 3; ++x)
    for (int y = 0; y < 2 - x; ++y)
      if (sg[o[y]] < sg[o[y + 1]]) {
        const int tmp = o[y];
        o[y] = o[y + 1];
        o[y + 1] = tmp;
      }
  double u[3][3];
  for (int c = 0; c < 3; ++c) {
    const int p = o[c];
    S[c] = sg[p];
    for (int r = 0; r < 3; ++r) {
      V[r * 3 + c] = v[r][p];
      u[r][c] = sg[p] > 0.0 ? a[r][p] / sg[p] : 0.0;
    }
  }
  // complete U where a singular value vanished (only the last two can)
  if (!(S[1] > 0.0)) {
    // pick any unit vector orthogonal to u0
    double e[3] = {0, 0, 0};
    const int ax = fabs(u[0][0]) < 0.577 ? 0 : (fabs(u[1][0]) < 0.577 ? 1 : 2);
    e[ax] = 1.0;
    const double d = e[0] * u[0][0] + e[1] * u[1][0] + e[2] * u[2][0];
    double n2 = 0;
    for (int r = 0; r < 3; ++r) {
      u[r][1] = e[r] - d * u[r][0];
      n2 += u[r][1] * u[r][1];
    }
    n2 = sqrt(n2);
    for (int r = 0; r < 3; ++r) u[r][1] /= n2;
  }
  if (!(S[2] > 0.0)) {
    u[0][2] = u[1][0] * u[2][1] - u[2][0] * u[1][1];
    u[1][2] = u[2][0] * u[0][1] - u[0][0] * u[2][1];
    u[2][2] = u[0][0] * u[1][1] - u[1][0] * u[0][1];
  }
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c) U[r * 3 + c] = u[r][c];
}

__device__ __forceinline__ double det3(const double* M) {
  return M[0] * (M[4] * M[8] - M[5] * M[7]) - M[1] * (M[3] * M[8] - M[5] * M[6]) +
         M[2] * (M[3] * M[7] - M[4] * M[6]);
}

// Nearest orthogonal matrix U V^T of R = U S V^T.
__device__ void polar3(const double* R, double* out) {
  double U[9], S[3], V[9];
  svd3(R, U, S, V);
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c)
      out[r * 3 + c] = U[r * 3] * V[c * 3] + U[r * 3 + 1] * V[c * 3 + 1] + U[r * 3 + 2] * V[c * 3 + 2];
}

// Derived float32 map and template mean for the current pose.
__device__ void refresh_pose(DevPose* ps, const DevStats* st) {
  for (int q = 0; q < 9; ++q) ps->A[q] = (float)(ps->s * ps->R[q]);
  for (int c = 0; c < 3; ++c) {
    ps->b[c] = (float)(ps->t[c] - st->xbar[c]);
    const double yb = ps->s * (st->ybar0[0] * ps->R[c] + st->ybar0[1] * ps->R[3 + c] +
                               st->ybar0[2] * ps->R[6 + c]) + ps->t[c];
    set_ybs(ps, c, yb - st->xbar[c]);
  }
}

__global__ void pose_init_kernel(DevPose* ps, const DevStats* st, int E) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  for (int q = 0; q < 9; ++q) ps->R[q] = (q % 4 == 0) ? 1.0 : 0.0;
  ps->t[0] = ps->t[1] = ps->t[2] = 0.0;
  ps->s = 1.0;
  ps->it = 0;
  ps->E = E;
  ps->degenerate = 0;
  refresh_pose(ps, st);
}

__global__ void pose_refresh_kernel(DevPose* ps, const DevStats* st) {
  if (threadIdx.x == 0 && blockIdx.x == 0) refresh_pose(ps, st);
}

cudaError_t launch_pose_init(Launch L, DevPose* pose, const DevStats* stats, int E) {
  pose_init_kernel<<<1, 32, 0, L.stream>>>(pose, stats, E);
  if (L.counter) ++*L.counter;
  return cudaGetLastError();
}

cudaError_t launch_pose_refresh(Launch L, DevPose* pose, const DevStats* stats) {
  pose_refresh_kernel<<<1, 32, 0, L.stream>>>(pose, stats);
  if (L.counter) ++*L.counter;
  return cudaGetLastError();
}

// ---- warp-parallel 3x3 algebra -------------------------------------------
// GB300 issues an FP64 warp instruction at a small fraction of the FP32 rate
// whatever the number of active lanes, so the finalize step spreads its 3x3
// matrices over a warp: lane l < 9 owns entry (l / 3, l % 3) (lanes 9..31
// mirror entry 8; their results are never stored).  A 3x3 product is then 3
// FP64 instructions for the warp instead of 27 for one thread.  Every
// function here must be called by all 32 lanes of the warp together.
constexpr unsigned WFULL = 0xffffffffu;

struct Lane3 {
  int q, r, c;
};
__device__ __forceinline__ Lane3 lane3() {
  const int q = min((int)(threadIdx.x & 31), 8);
  return {q, q / 3, q % 3};
}
__device__ __forceinline__ double wget(double v, int idx) { return __shfl_sync(WFULL, v, idx); }

// (A B)_rc and (A^T B)_rc for lane-owned A and B
__device__ __forceinline__ double wmul(double a, double b, Lane3 L) {
  const double acc = wget(a, L.r * 3) * wget(b, L.c);
  return fma(wget(a, L.r * 3 + 2), wget(b, 6 + L.c), fma(wget(a, L.r * 3 + 1), wget(b, 3 + L.c), acc));
}
__device__ __forceinline__ double wmul_ta(double a, double b, Lane3 L) {
  const double acc = wget(a, L.r) * wget(b, L.c);
  return fma(wget(a, 6 + L.r), wget(b, 6 + L.c), fma(wget(a, 3 + L.r), wget(b, 3 + L.c), acc));
}

// Sum and maximum over lanes 0..8, the same value in every lane (lane 0's).
__device__ __forceinline__ float wsum9(float v) {
  if ((threadIdx.x & 31) >= 9) v = 0.f;
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(WFULL, v, off);
  return __shfl_sync(WFULL, v, 0);
}
__device__ __forceinline__ double wsum9d(double v) {
  if ((threadIdx.x & 31) >= 9) v = 0.0;
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(WFULL, v, off);
  return __shfl_sync(WFULL, v, 0);
}
__device__ __forceinline__ float wmax9(float v) {
  if ((threadIdx.x & 31) >= 9) v = 0.f;
  for (int off = 16; off > 0; off >>= 1) v = fmaxf(v, __shfl_xor_sync(WFULL, v, off));
  return __shfl_sync(WFULL, v, 0);
}

// 1/x for x > 0 in float64 from the float32 reciprocal and two Newton steps.
__device__ __forceinline__ double wrcp(double x) {
  double r = (double)(1.0f / (float)x);
  r = fma(r, fma(-x, r, 1.0), r);
  return fma(r, fma(-x, r, 1.0), r);
}

// Orthogonal polar factor Q of A (A = Q H, H symmetric positive definite)
// for det A > 0 by Newton's iteration X <- (g X + X^-T / g) / 2 with
// Frobenius-norm scaling g = (|X^-1| / |X|)^(1/2) while far from the limit
// (Higham, "Computing the polar decomposition -- with applications", 1986),
// in float64 with the 3x3 spread over the warp: Q's entry in each lane.
// X^-T is the cofactor matrix over the determinant.  The input is first
// scaled to unit Frobenius norm, which leaves the polar factor unchanged and
// keeps the FP32 norms below in range.  The scaling factor g and the stop
// test use FP32 sums: any positive weights (a X + b X^-T) / 2 keep the polar
// factor, so they only steer convergence; the last steps use a = b = 1
// exactly.  Returns false (the caller then takes the SVD) when det A <= 0,
// when |A|_F |A^-1|_F > 1e6, or when the iteration has not settled in 40
// steps.
__device__ bool polar_newton_warp(double A, Lane3 L, double& Q) {
  const double n2 = wsum9d(A * A);
  if (!(n2 > 0.0) || !isfinite(n2)) return false;
  double X = A * (1.0 / sqrt(n2));
  const int r1 = (L.r + 1) % 3, r2 = (L.r + 2) % 3, c1 = (L.c + 1) % 3, c2 = (L.c + 2) % 3;
  bool scale = true;
  for (int it = 0; it < 40; ++it) {
    double C = fma(-wget(X, r1 * 3 + c2), wget(X, r2 * 3 + c1), wget(X, r1 * 3 + c1) * wget(X, r2 * 3 + c2));
    const double det = fma(wget(X, 2), wget(C, 2), fma(wget(X, 1), wget(C, 1), wget(X, 0) * wget(C, 0)));
    if (!(det > 1e-30) || !isfinite(det)) return false;
    C *= wrcp(det);  // X^-T
    const float fx = (float)X, fc = (float)C;
    const float nx = wsum9(fx * fx), ny = wsum9(fc * fc);
    if (it == 0 && !(nx * ny <= 1e12f)) return false;
    const float g = scale ? sqrtf(sqrtf(ny / nx)) : 1.f;
    const double Xn = fma(0.5 * (double)g, X, (double)(0.5f / g) * C);
    const float dx = (float)(Xn - X), fn = (float)Xn;
    const float dd = wsum9(dx * dx), nn = wsum9(fn * fn);
    X = Xn;
    // stop once a step changed X by at most 1e-9 of its norm: Newton's
    // iteration converges quadratically there, so this iterate is within
    // about (1e-9)^2 of the polar factor, below float64 rounding
    if (dd <= 1e-18f * nn) break;
    scale = dd > 1e-4f * nn;
    if (it == 39) return false;
  }
  Q = X;
  return true;
}

// Polar factor of A (lane-owned) with most of the work in float32.  On
// GB300 a float64 instruction costs about 65 cycles whatever the number of
// active lanes, and consecutive ones do not overlap, so the float64 work is
// kept to the few products that need it.  Every lane first runs the same
// scaled Newton iteration on its own float copy X of the 3x3, then two
// corrections against A itself bring the factor to float64 accuracy.  A
// correction writes the current factor as Q = R (I + S), R orthogonal and
// S = (Q^T Q - I) / 2 symmetric and small, forms B = Q^T A (float64), so
// that R^T A = (I - S) B to first order, and takes the small rotation w that
// makes R (I + [w]x)'s transpose times A symmetric: with H = (B + B^T) / 2
// and k = axial of the skew part of (I - S) B doubled, the symmetric-H
// identity [w]x H + H [w]x = [(tr(H) I - H) w]x gives (tr(H) I - H) w = k.
// Then Q <- Q + X ([w]x - S).  Only Q^T Q, Q^T A, B - B^T and the final
// sum are float64; the rest are small quantities whose float32 rounding is
// second order.  Each correction squares the error (float32's ~1e-7, then
// float64 rounding).  Returns false, and the caller takes polar_newton_warp,
// for inputs out of float32 range, det <= 0, a Frobenius condition estimate
// above 1e3, or a correction that does not shrink.
__device__ bool polar_float_refined_warp(double A, Lane3 L, double& Q) {
  const float fa = (float)A;
  float x[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) x[k] = __shfl_sync(WFULL, fa, k);
  float n2 = 0.f;
#pragma unroll
  for (int k = 0; k < 9; ++k) n2 = fmaf(x[k], x[k], n2);
  if (!(n2 > 0.f) || !isfinite(n2)) return false;
  const float inv = rsqrtf(n2);
#pragma unroll
  for (int k = 0; k < 9; ++k) x[k] *= inv;
  bool scale = true, done = false;
  for (int it = 0; it < 20 && !done; ++it) {
    float c[9];  // cofactors of X, then X^-T
    c[0] = x[4] * x[8] - x[5] * x[7];
    c[1] = x[5] * x[6] - x[3] * x[8];
    c[2] = x[3] * x[7] - x[4] * x[6];
    c[3] = x[2] * x[7] - x[1] * x[8];
    c[4] = x[0] * x[8] - x[2] * x[6];
    c[5] = x[1] * x[6] - x[0] * x[7];
    c[6] = x[1] * x[5] - x[2] * x[4];
    c[7] = x[2] * x[3] - x[0] * x[5];
    c[8] = x[0] * x[4] - x[1] * x[3];
    const float det = fmaf(x[2], c[2], fmaf(x[1], c[1], x[0] * c[0]));
    if (!(det > 1e-20f) || !isfinite(det)) return false;
    const float rd = __frcp_rn(det);
    float nx = 0.f, ny = 0.f;
#pragma unroll
    for (int k = 0; k < 9; ++k) {
      c[k] *= rd;
      nx = fmaf(x[k], x[k], nx);
      ny = fmaf(c[k], c[k], ny);
    }
    if (it == 0 && !(nx * ny <= 1e6f)) return false;
    const float g = scale ? sqrtf(sqrtf(__fdividef(ny, nx))) : 1.f;
    const float a = 0.5f * g, b = __fdividef(0.5f, g);
    float dd = 0.f, nn = 0.f;
#pragma unroll
    for (int k = 0; k < 9; ++k) {
      const float xn = fmaf(a, x[k], b * c[k]);
      const float d = xn - x[k];
      dd = fmaf(d, d, dd);
      nn = fmaf(xn, xn, nn);
      x[k] = xn;
    }
    done = dd <= 1e-10f * nn;
    scale = dd > 1e-4f * nn;
  }
  if (!done) return false;
  const int q = L.q;
  float mine = x[0];
#pragma unroll
  for (int k = 1; k < 9; ++k) mine = (q == k) ? x[k] : mine;
  double Qd = (double)mine;
  // A scaled by a power of two near 1 / ||A|| (exact), so that the 3x3
  // quantities below stay near unit size
  int e2 = 0;
  frexpf(sqrtf(n2), &e2);
  const double As = A * __longlong_as_double((long long)(1023 - e2) << 52);
  const double I = (L.r == L.c) ? 1.0 : 0.0;
  for (int step = 0; step < 2; ++step) {
    const double E = wmul_ta(Qd, Qd, L) - I;
    const double B = wmul_ta(Qd, As, L);
    const double K = B - wget(B, L.c * 3 + L.r);
    const float ef = (float)E, bf = (float)B, kf = (float)K;
    float sm[9], bm[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) {
      sm[k] = 0.5f * __shfl_sync(WFULL, ef, k);
      bm[k] = __shfl_sync(WFULL, bf, k);
    }
    const float k21 = __shfl_sync(WFULL, kf, 7), k02 = __shfl_sync(WFULL, kf, 2), k10 = __shfl_sync(WFULL, kf, 3);
    // entries of S B for its skew part
    auto sb = [&](int r, int c) { return fmaf(sm[r * 3 + 2], bm[6 + c], fmaf(sm[r * 3 + 1], bm[3 + c], sm[r * 3] * bm[c])); };
    const float kp0 = k21 - (sb(2, 1) - sb(1, 2));
    const float kp1 = k02 - (sb(0, 2) - sb(2, 0));
    const float kp2 = k10 - (sb(1, 0) - sb(0, 1));
    // M = tr(H) I - H, H = (B + B^T) / 2
    const float tr = bm[0] + bm[4] + bm[8];
    const float m00 = tr - bm[0], m11 = tr - bm[4], m22 = tr - bm[8];
    const float m01 = -0.5f * (bm[1] + bm[3]), m02 = -0.5f * (bm[2] + bm[6]), m12 = -0.5f * (bm[5] + bm[7]);
    // adj(M) (symmetric) and det M
    const float a00 = m11 * m22 - m12 * m12, a01 = m02 * m12 - m01 * m22, a02 = m01 * m12 - m02 * m11;
    const float a11 = m00 * m22 - m02 * m02, a12 = m01 * m02 - m00 * m12, a22 = m00 * m11 - m01 * m01;
    const float detM = fmaf(m02, a02, fmaf(m01, a01, m00 * a00));
    if (!(detM > 0.f) || !isfinite(detM)) return false;
    const float rdm = __frcp_rn(detM);
    const float w0 = rdm * fmaf(a02, kp2, fmaf(a01, kp1, a00 * kp0));
    const float w1 = rdm * fmaf(a12, kp2, fmaf(a11, kp1, a01 * kp0));
    const float w2 = rdm * fmaf(a22, kp2, fmaf(a12, kp1, a02 * kp0));
    const float wn = fmaf(w2, w2, fmaf(w1, w1, w0 * w0));
    if (!(wn <= (step == 0 ? 1e-8f : 1e-20f))) return false;
    // D = [w]x - S, and this lane's entry of X D
    const float d[9] = {-sm[0],      -w2 - sm[1], w1 - sm[2],  w2 - sm[3], -sm[4],
                        -w0 - sm[5], -w1 - sm[6], w0 - sm[7], -sm[8]};
    float p = 0.f;
#pragma unroll
    for (int k = 0; k < 9; ++k) {
      const float xd = fmaf(x[(k / 3) * 3 + 2], d[6 + k % 3], fmaf(x[(k / 3) * 3 + 1], d[3 + k % 3], x[(k / 3) * 3] * d[k % 3]));
      p = (q == k) ? xd : p;
    }
    Qd += (double)p;
  }
  Q = Qd;
  return true;
}

// Warp form of reorthonormalise for the product of the pose's rotation and
// the increment, both orthogonal to float64 rounding: one Newton-Schulz step
// brings R^T R - I back to rounding (a second changes nothing above it);
// false (the caller takes the SVD route) when R^T R is further than 1e-6
// from I.
__device__ bool reorth_warp(double R, Lane3 L, double& out) {
  const double I = (L.r == L.c) ? 1.0 : 0.0;
  const double e = wmul_ta(R, R, L) - I;
  if (!(wmax9(fabsf((float)e)) <= 1e-6f)) return false;
  out = wmul(R, fma(-0.5, e, I), L);
  return true;
}

// Column sums of the per-block partials.  A float64 instruction costs about
// 65 cycles on GB300 whatever the number of active lanes, and dependent ones
// do not overlap, so the sums are arranged by the length of the dependent
// chain in one lane (lane q < 13 adds column q):
// * up to FINALIZE_WARP_ROWS rows, warp 0 adds them alone, in order;
// * up to FINALIZE_SPLIT_ROWS, each of the 8 warps adds every 8th row (warp
//   w: rows w, w + 8, ...) and warp 0 adds the 8 warp sums in order, a chain
//   of rows / 8 + 8 additions instead of rows;
// * beyond that, each thread adds its rows and a block-wide tree follows
//   (about 150 float64 instructions however many rows there are).
constexpr int FINALIZE_WARP_ROWS = 16;
constexpr int FINALIZE_SPLIT_ROWS = 512;

// Warp 0 forms the update from the 13 totals v (the same in every lane of
// warp 0; F[3], W, T[3][3]); lane (r, c) owns entry (r, c) of each 3x3.
// sh is scratch (at least 64 doubles).
__device__ void finalize_update(const double (&v)[13], DevPose* ps, const DevStats* __restrict__ st,
                                StepParams sp, int* err, double (*sh)[RED_THREADS]) {
  const Lane3 L = lane3();
  const int lane = threadIdx.x;
  const double W = v[3];
  const double Tq = v[4 + L.q];  // T[a][b] = sum_i f_i[a] (Y_i - ybar)[b]
  const int it = ps->it;
  const double E = (double)ps->E;
  // Eq. 12, 0-based iteration index: G / G1 = 0.1 + 0.9 / (1 + e), written
  // over one division (each float64 division is a chain of about ten
  // float64 instructions, about 65 cycles each on GB300)
  const double e1 = 1.0 + exp(-((double)it - E / 2.0));
  const double gnum = fma(0.1, e1, 0.9);  // (G / G1) (1 + e)
  double kappa, dq;                       // dc = dq v_c
  bool bad = false;
  if (sp.step_mode == 0) {
    // kappa = eta0 (G / G1) M / W, and Eq. 5.5's d = kappa v / M needs no M
    if (!(W > 0.0) || !isfinite(W)) bad = true;
    dq = bad ? 0.0 : sp.eta0 * gnum / (e1 * W);
    kappa = dq * (double)sp.M;
  } else {
    kappa = sp.G1 * gnum / e1 * sp.time * sp.time;
    dq = kappa / (double)sp.M;
  }
  const double s = ps->s;
  const double Rq = ps->R[L.q];
  // template mean at this pose, component L.c in each lane, and t - ybar
  const double tc = ps->t[L.c];
  const double ybc =
      fma(s, fma(st->ybar0[2], ps->R[6 + L.c], fma(st->ybar0[1], ps->R[3 + L.c], st->ybar0[0] * ps->R[L.c])), tc);
  const double tmy = tc - ybc;
  const double dc = dq * v[L.c];  // Eq. 5.5, unit masses, v = 0 (component c)
  // C^ = Y_D^T Y_c = s^2 R^T S0 R + kappa T   (Eq. 6 with the displaced cloud)
  const double SR = wmul(st->S0[L.q], Rq, L);
  const double Ch = fma(kappa, Tq, s * s * wmul_ta(Rq, SR, L));
  bad = bad || !isfinite(Ch) || !isfinite(dc);
  if (__any_sync(WFULL, bad)) {
    if (lane == 0) {
      atomicOr(err, ERR_NUMERIC);
      ps->it = it + 1;
    }
    return;
  }
  // Eq. 6: C^ = U S V^T, dd = sign det(V U^T), R_inc = V diag(1, 1, dd) U^T.
  // For det C^ > 0 (dd = 1) that is Q^T, Q the orthogonal polar factor of C^
  // (C^ = (U V^T)(V S V^T)), taken by Newton's iteration (in float32 with
  // float64 corrections, else all in float64); the SVD handles det C^ <= 0,
  // near-singular C^ and the degenerate case.
  double Rinc, Qp;
  if (polar_float_refined_warp(Ch, L, Qp) || polar_newton_warp(Ch, L, Qp)) {
    Rinc = wget(Qp, L.c * 3 + L.r);
  } else {
    double* scr = &sh[0][0];
    if (lane < 9) scr[lane] = Ch;
    __syncwarp();
    if (lane == 0) {
      double U[9], Sg[3], V[9], Ri[9];
      svd3(scr, U, Sg, V);
      if (!(Sg[0] > 0.0) || Sg[1] <= 1e-12 * Sg[0]) {
        for (int q = 0; q < 9; ++q) Ri[q] = (q % 4 == 0) ? 1.0 : 0.0;
        ps->degenerate += 1;
      } else {
        const double dd = (det3(V) * det3(U)) >= 0.0 ? 1.0 : -1.0;
        const double D[3] = {1.0, 1.0, dd};
        for (int r = 0; r < 3; ++r)
          for (int c = 0; c < 3; ++c)
            Ri[r * 3 + c] = V[r * 3] * D[0] * U[c * 3] + V[r * 3 + 1] * D[1] * U[c * 3 + 1] +
                            V[r * 3 + 2] * D[2] * U[c * 3 + 2];
      }
      for (int q = 0; q < 9; ++q) scr[16 + q] = Ri[q];
    }
    __syncwarp();
    Rinc = scr[16 + L.q];
  }
  // scale model (Sec. III-B): c from the largest covariance eigenvalues
  const double eY = s * s * st->eY0;
  double cs = 1.0;
  if (sp.scale_mode == 0) cs = sqrt(st->eX / eY);
  else if (sp.scale_mode == 1) cs = st->eX / eY;
  // Eq. 8, Eq. 9: Y(t+1) = c (Y - ybar) R_inc + ybar + d, composed into the pose
  // (lanes 0, 1, 2 hold t - ybar of components 0, 1, 2)
  double acc = wget(tmy, 0) * wget(Rinc, L.c);
  acc = fma(wget(tmy, 1), wget(Rinc, 3 + L.c), acc);
  acc = fma(wget(tmy, 2), wget(Rinc, 6 + L.c), acc);
  const double tn = fma(cs, acc, ybc + dc);  // component c
  const double RR = wmul(Rq, Rinc, L);
  double Rn;
  if (!reorth_warp(RR, L, Rn)) {
    double* scr = &sh[0][0];
    if (lane < 9) scr[32 + lane] = RR;
    __syncwarp();
    if (lane == 0) polar3(scr + 32, scr + 48);
    __syncwarp();
    Rn = scr[48 + L.q];
  }
  const bool ok = isfinite(cs) && isfinite(Rn) && isfinite(tn);
  if (!__all_sync(WFULL, ok)) {
    if (lane == 0) {
      atomicOr(err, ERR_NUMERIC);
      ps->it = it + 1;
    }
    return;
  }
  // new pose and its derived float32 map (the warp form of refresh_pose)
  const double sn = cs * s;
  const double ybs = fma(sn, fma(st->ybar0[2], wget(Rn, 6 + L.c), fma(st->ybar0[1], wget(Rn, 3 + L.c),
                                                                         st->ybar0[0] * wget(Rn, L.c))),
                         tn) - st->xbar[L.c];
  if (lane < 9) {
    ps->R[lane] = Rn;
    ps->A[lane] = (float)(sn * Rn);
  }
  if (lane < 3) {
    ps->t[lane] = tn;
    ps->b[lane] = (float)(tn - st->xbar[lane]);
    set_ybs(ps, lane, ybs);
  }
  if (lane == 0) {
    ps->s = sn;
    ps->it = it + 1;
  }
}

// Totals of nblocks rows of 13 partials (fixed order), then the update.
__device__ void finalize_body(const double* __restrict__ blockpart, int nblocks, DevPose* ps,
                              const DevStats* __restrict__ st, StepParams sp, int* err,
                              double (*sh)[RED_THREADS]) {
  double v[13];
  if (nblocks <= FINALIZE_WARP_ROWS) {
    if (threadIdx.x >= 32) return;
    const int lane = threadIdx.x;
    double col = 0.0;
    if (lane < 13)
      for (int b = 0; b < nblocks; ++b) col += blockpart[(size_t)b * 13 + lane];
#pragma unroll
    for (int q = 0; q < 13; ++q) v[q] = __shfl_sync(WFULL, col, q);
  } else if (nblocks <= FINALIZE_SPLIT_ROWS) {
    constexpr int NW = RED_THREADS / 32;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    double col = 0.0;
    if (lane < 13)
      for (int b = warp; b < nblocks; b += NW) col += blockpart[(size_t)b * 13 + lane];
    if (lane < 13) sh[lane][warp] = col;
    __syncthreads();
    if (threadIdx.x >= 32) return;
    double tot = 0.0;
    if (lane < 13)
      for (int k = 0; k < NW; ++k) tot += sh[lane][k];
    __syncwarp();  // every lane has read its sums: sh is scratch from here on
#pragma unroll
    for (int q = 0; q < 13; ++q) v[q] = __shfl_sync(WFULL, tot, q);
  } else {
#pragma unroll
    for (int q = 0; q < 13; ++q) v[q] = 0.0;
    for (int bidx = threadIdx.x; bidx < nblocks; bidx += RED_THREADS) {
#pragma unroll
      for (int q = 0; q < 13; ++q) v[q] += blockpart[(size_t)bidx * 13 + q];
    }
    block_sum<13>(v, sh);
    __syncthreads();  // every thread has read the totals: sh is scratch from here on
    if (threadIdx.x >= 32) return;
  }
  finalize_update(v, ps, st, sp, err, sh);
}

// Combine and finalize in one block, for templates of at most
// FUSED_MAX_SLOTS padded slots (the latency regime of small problems).
// 1. FUSED_THREADS threads form the points' (f, W_i) from their split
//    partials (point_fw) into shared memory: a thread's points are
//    sequential trips to memory, so more threads than the sums below use
//    shorten that chain.
// 2. The first RED_THREADS threads add them up (thread t: points t,
//    t + RED_THREADS, ... in order, through point_acc), the order a
//    RED_THREADS-thread pass over the points would take.
// 3. The 13 sums are reduced per warp (float64) and across the warps in
//    order by warp 0, and warp 0 updates the pose.
// One launch per iteration instead of two, and no per-block partials.
constexpr int FUSED_THREADS = 512;

__global__ void __launch_bounds__(FUSED_THREADS, 1)
    combine_finalize_kernel(const float4* __restrict__ partial, int S, int mpad, int m,
                            const float4* __restrict__ Y0r, const float* __restrict__ aY32, int g_mode,
                            DevPose* ps, const DevStats* __restrict__ st, StepParams sp, int* err) {
  // (f, W_i) per point in steps 1-2; the float64 sums and scratch from step 3
  __shared__ __align__(16) unsigned char smem[FUSED_MAX_SLOTS * sizeof(float4)];
  static_assert(FUSED_MAX_SLOTS * sizeof(float4) >= sizeof(double) * 13 * RED_THREADS, "scratch too small");
  float4* fws = reinterpret_cast<float4*>(smem);
  double(*sh)[RED_THREADS] = reinterpret_cast<double(*)[RED_THREADS]>(smem);
  const PointFrame fr(ps);
  for (int i = threadIdx.x; i < m; i += FUSED_THREADS)
    fws[i] = point_fw(partial, (size_t)mpad, S, i, Y0r[i], g_mode == 1 ? aY32[i] : 1.f, fr);
  __syncthreads();
  if (threadIdx.x >= RED_THREADS) return;  // all of ps read
  float acc[13];
#pragma unroll
  for (int q = 0; q < 13; ++q) acc[q] = 0.f;
  for (int i = threadIdx.x; i < m; i += RED_THREADS) point_acc(fws[i], Y0r[i], fr, acc);
  double w[16];
#pragma unroll
  for (int q = 0; q < 13; ++q) w[q] = (double)acc[q];
  w[13] = w[14] = w[15] = 0.0;
  warp_reduce16(w);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  __syncthreads();  // every (f, W_i) read: smem holds the float64 sums from here
  // even lanes hold quantities 0..15 after the reduction; 13..15 are padding
  // and have no row in sh
  if ((lane & 1) == 0) {
    const int q = warp_reduce16_slot(lane);
    if (q < 13) sh[q][warp] = w[0];
  }
  __syncthreads();  // all of ps and sh read/written: warp 0 updates the pose from here
  if (warp != 0) return;
  double col = 0.0;
  if (lane < 13)
    for (int k = 0; k < RED_THREADS / 32; ++k) col += sh[lane][k];
  __syncwarp();
  double v[13];
#pragma unroll
  for (int q = 0; q < 13; ++q) v[q] = __shfl_sync(WFULL, col, q);
  finalize_update(v, ps, st, sp, err, sh);
}

cudaError_t launch_combine_finalize(Launch L, const float4* partial, int S, int mpad, int m, const float4* Y0r,
                                    const float* aY32, int g_mode, DevPose* pose, const DevStats* stats,
                                    StepParams sp, int* err) {
  combine_finalize_kernel<<<1, FUSED_THREADS, 0, L.stream>>>(partial, S, mpad, m, Y0r, aY32, g_mode, pose, stats,
                                                             sp, err);
  if (L.counter) ++*L.counter;
  return cudaGetLastError();
}

__global__ void __launch_bounds__(RED_THREADS)
    finalize_kernel(const double* __restrict__ blockpart, int nblocks, DevPose* ps,
                    const DevStats* __restrict__ st, StepParams sp, int* err) {
  __shared__ double sh[13][RED_THREADS];
  finalize_body(blockpart, nblocks, ps, st, sp, err, sh);
}

// One block per pair of a batch.
__global__ void __launch_bounds__(RED_THREADS)
    finalize_multi_kernel(const double* __restrict__ blockpart, const BatchPair* __restrict__ pairs,
                          DevPose* poses, const DevStats* __restrict__ stats, StepParams sp, int* err) {
  __shared__ double sh[13][RED_THREADS];
  const BatchPair& bp = pairs[blockIdx.x];
  StepParams spp = sp;
  spp.M = (int)bp.m;
  finalize_body(blockpart + (size_t)bp.cblk0 * 13, bp.ncblk, poses + blockIdx.x, stats + blockIdx.x, spp, err, sh);
}

cudaError_t launch_finalize_multi(Launch L, const double* blockpart, const BatchPair* pairs, int npairs,
                                  DevPose* poses, const DevStats* stats, StepParams sp, int* err) {
  finalize_multi_kernel<<<npairs, RED_THREADS, 0, L.stream>>>(blockpart, pairs, poses, stats, sp, err);
  if (L.counter) ++*L.counter;
  return cudaGetLastError();
}

__global__ void pose_init_multi_kernel(DevPose* poses, const DevStats* stats, int npairs, int E) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= npairs) return;
  DevPose* ps = poses + p;
  for (int q = 0; q < 9; ++q) ps->R[q] = (q % 4 == 0) ? 1.0 : 0.0;
  ps->t[0] = ps->t[1] = ps->t[2] = 0.0;
  ps->s = 1.0;
  ps->it = 0;
  ps->E = E;
  ps->degenerate = 0;
  refresh_pose(ps, stats + p);
}

cudaError_t launch_pose_init_multi(Launch L, DevPose* poses, const DevStats* stats, int npairs, int E) {
  pose_init_multi_kernel<<<(npairs + 127) / 128, 128, 0, L.stream>>>(poses, stats, npairs, E);
  if (L.counter) ++*L.counter;
  return cudaGetLastError();
}

cudaError_t launch_finalize(Launch L, const double* blockpart, int nblocks, DevPose* pose,
                            const DevStats* stats, StepParams sp, int* err) {
  finalize_kernel<<<1, RED_THREADS, 0, L.stream>>>(blockpart, nblocks, pose, stats, sp, err);
  if (L.counter) ++*L.counter;
  return cudaGetLastError();
}

// moved = s Y0 R + t (Eq. 9), float64 arithmetic, float32 output [m][3]
__global__ void apply_kernel(const float4* __restrict__ Y4, int m, const DevPose* __restrict__ ps,
                             float* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m) return;
  const float4 y = Y4[i];
  for (int c = 0; c < 3; ++c) {
    const double v = ps->s * ((double)y.x * ps->R[c] + (double)y.y * ps->R[3 + c] +
                              (double)y.z * ps->R[6 + c]) + ps->t[c];
    out[(size_t)i * 3 + c] = (float)v;
  }
}

cudaError_t launch_apply(Launch L, const float4* Y4, int m, const DevPose* pose, float* out) {
  if (m <= 0) return cudaSuccess;
  apply_kernel<<<(m + 255) / 256, 256, 0, L.stream>>>(Y4, m, pose, out);
  if (L.counter) ++*L.counter;
  return cudaGetLastError();
}

}  // namespace scgr
