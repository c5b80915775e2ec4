// Pose update in float64 (Eq. 5.5, Eq. 6, Eq. 8, Eq. 9, Eq. 12): one block
// reduces the per-block (F, W, T) partials in a fixed order, then one thread
// forms the step, the Kabsch rotation by a one-sided Jacobi SVD, the scale,
// the composed pose and its polar re-orthonormalisation.  The pose never
// leaves the device, so a run of iterations is a plain sequence of launches.
#include <cmath>

#include "common.cuh"

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

// Z = X Y (3x3 row-major)
__device__ __forceinline__ void mul3(const double* X, const double* Y, double* Z) {
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c) Z[r * 3 + c] = X[r * 3] * Y[c] + X[r * 3 + 1] * Y[3 + c] + X[r * 3 + 2] * Y[6 + c];
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
    ps->ybs[c] = yb - st->xbar[c];
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

__device__ void finalize_body(const double* __restrict__ blockpart, int nblocks, DevPose* ps,
                              const DevStats* __restrict__ st, StepParams sp, int* err,
                              double (*sh)[RED_THREADS]) {
  double v[13];
#pragma unroll
  for (int q = 0; q < 13; ++q) v[q] = 0.0;
  for (int bidx = threadIdx.x; bidx < nblocks; bidx += RED_THREADS) {
#pragma unroll
    for (int q = 0; q < 13; ++q) v[q] += blockpart[(size_t)bidx * 13 + q];
  }
  block_sum<13>(v, sh);
  if (threadIdx.x != 0) return;

  const double F[3] = {v[0], v[1], v[2]};
  const double W = v[3];
  const double* T = v + 4;  // T[a][b] = sum_i f_i[a] (Y_i - ybar)[b]
  const int it = ps->it;
  const double E = (double)ps->E;
  // Eq. 12, 0-based iteration index
  const double G = 0.1 * sp.G1 + 0.9 * sp.G1 / (1.0 + exp(-((double)it - E / 2.0)));
  double kappa;
  bool bad = false;
  if (sp.step_mode == 0) {
    if (!(W > 0.0) || !isfinite(W)) bad = true;
    kappa = bad ? 0.0 : sp.eta0 * (G / sp.G1) * (double)sp.M / W;
  } else {
    kappa = G * sp.time * sp.time;
  }
  const double s = ps->s;
  const double* R = ps->R;
  double d[3], ybar[3];
  for (int c = 0; c < 3; ++c) {
    d[c] = kappa * F[c] / (double)sp.M;  // Eq. 5.5, unit masses, v = 0
    ybar[c] = s * (st->ybar0[0] * R[c] + st->ybar0[1] * R[3 + c] + st->ybar0[2] * R[6 + c]) + ps->t[c];
  }
  // C^ = Y_D^T Y_c = s^2 R^T S0 R + kappa T   (Eq. 6 with the displaced cloud)
  double SR[9], Syy[9], Ch[9];
  mul3(st->S0, R, SR);
  for (int a = 0; a < 3; ++a)
    for (int b2 = 0; b2 < 3; ++b2) {
      double acc = 0.0;
      for (int r = 0; r < 3; ++r) acc += R[r * 3 + a] * SR[r * 3 + b2];
      Syy[a * 3 + b2] = s * s * acc;
    }
  for (int q = 0; q < 9; ++q) Ch[q] = Syy[q] + kappa * T[q];
  for (int q = 0; q < 9; ++q)
    if (!isfinite(Ch[q])) bad = true;
  for (int c = 0; c < 3; ++c)
    if (!isfinite(d[c])) bad = true;
  if (bad) {
    atomicOr(err, ERR_NUMERIC);
    ps->it = it + 1;
    return;
  }
  // Eq. 6: C^ = U S V^T, dd = sign det(V U^T), R_inc = V diag(1, 1, dd) U^T
  double U[9], Sg[3], V[9], Rinc[9];
  svd3(Ch, U, Sg, V);
  if (!(Sg[0] > 0.0) || Sg[1] <= 1e-12 * Sg[0]) {
    for (int q = 0; q < 9; ++q) Rinc[q] = (q % 4 == 0) ? 1.0 : 0.0;
    ps->degenerate += 1;
  } else {
    const double dd = (det3(V) * det3(U)) >= 0.0 ? 1.0 : -1.0;
    const double D[3] = {1.0, 1.0, dd};
    for (int r = 0; r < 3; ++r)
      for (int c = 0; c < 3; ++c)
        Rinc[r * 3 + c] = V[r * 3] * D[0] * U[c * 3] + V[r * 3 + 1] * D[1] * U[c * 3 + 1] +
                          V[r * 3 + 2] * D[2] * U[c * 3 + 2];
  }
  // scale model (Sec. III-B): c from the largest covariance eigenvalues
  const double eY = s * s * st->eY0;
  double cs = 1.0;
  if (sp.scale_mode == 0) cs = sqrt(st->eX / eY);
  else if (sp.scale_mode == 1) cs = st->eX / eY;
  // Eq. 8, Eq. 9: Y(t+1) = c (Y - ybar) R_inc + ybar + d, composed into the pose
  double tn[3];
  for (int c = 0; c < 3; ++c) {
    double acc = 0.0;
    for (int r = 0; r < 3; ++r) acc += (ps->t[r] - ybar[r]) * Rinc[r * 3 + c];
    tn[c] = cs * acc + ybar[c] + d[c];
  }
  double RR[9], Rn[9];
  mul3(R, Rinc, RR);
  polar3(RR, Rn);
  bool ok = isfinite(cs);
  for (int q = 0; q < 9; ++q) ok = ok && isfinite(Rn[q]);
  for (int c = 0; c < 3; ++c) ok = ok && isfinite(tn[c]);
  if (!ok) {
    atomicOr(err, ERR_NUMERIC);
    ps->it = it + 1;
    return;
  }
  for (int q = 0; q < 9; ++q) ps->R[q] = Rn[q];
  for (int c = 0; c < 3; ++c) ps->t[c] = tn[c];
  ps->s = cs * s;
  ps->it = it + 1;
  refresh_pose(ps, st);
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
