// One-time descriptor pass (Sec. III-A, Sec. IV): input packing and
// validation, k-nearest neighbours, curvature, cloud statistics of the scale
// model (Sec. III-B), sigma of Eq. 3, and the records the force kernel reads.
#include <cmath>
#include <climits>

#include "common.cuh"

namespace scgr {

static inline cudaError_t after_launch(Launch L) {
  if (L.counter) ++*L.counter;
  return cudaGetLastError();
}

// ---- pack + validate ----------------------------------------------------
__global__ void pack_kernel(const float* __restrict__ xyz, int64_t n, float4* __restrict__ out,
                            int* __restrict__ err) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  float x = xyz[3 * i], y = xyz[3 * i + 1], z = xyz[3 * i + 2];
  // |x| <= 1e18 keeps every squared-distance key finite in float32
  const bool ok = isfinite(x) && isfinite(y) && isfinite(z) && fabsf(x) <= 1e18f &&
                  fabsf(y) <= 1e18f && fabsf(z) <= 1e18f;
  if (!ok) {
    atomicOr(err, ERR_NONFINITE);
    x = y = z = 0.f;
  }
  out[i] = make_float4(x, y, z, 0.f);
}

cudaError_t launch_pack(Launch L, const float* xyz, int64_t n, float4* out, int* err) {
  if (n <= 0) return cudaSuccess;
  const int tpb = 256;
  pack_kernel<<<(unsigned)((n + tpb - 1) / tpb), tpb, 0, L.stream>>>(xyz, n, out, err);
  return after_launch(L);
}

// ---- brute-force kNN ----------------------------------------------------
// Each thread owns one query and keeps its KC best (key, index) pairs sorted
// in registers.  Candidates are scanned in increasing index order, so a
// candidate whose key equals the current KC-th key never displaces it: ties
// go to the lower index.  The key is the float32 value
// (dx*dx + dy*dy) + dz*dz with every operation rounded on its own
// (__fmul_rn / __fadd_rn forbid contraction into fused multiply-adds).
constexpr int KNN_TPB = 128;
constexpr int KNN_TILE = 1024;

// Insert (key, idx) into the sorted list kd/ki of KC entries if it beats the
// KC-th key; a key equal to an entry stays behind it (candidates arrive in
// increasing index order, so ties keep the lower index first).
template <int KC>
__device__ __forceinline__ void knn_insert(float key, int idx, float* kd, int* ki) {
  if (key < kd[KC - 1]) {
    kd[KC - 1] = key;
    ki[KC - 1] = idx;
#pragma unroll
    for (int m = KC - 1; m > 0; --m) {
      if (kd[m] < kd[m - 1]) {
        const float tk = kd[m];
        kd[m] = kd[m - 1];
        kd[m - 1] = tk;
        const int ti = ki[m];
        ki[m] = ki[m - 1];
        ki[m - 1] = ti;
      }
    }
  }
}

__device__ __forceinline__ float knn_key(float4 q, float4 c) {
  const float dx = __fsub_rn(q.x, c.x);
  const float dy = __fsub_rn(q.y, c.y);
  const float dz = __fsub_rn(q.z, c.z);
  return __fadd_rn(__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)), __fmul_rn(dz, dz));
}

// Candidates that beat the KC-th key wait in a short per-thread queue; the
// warp merges all queues into the sorted lists together once any queue could
// overflow.  Inserting at once costs a 16-step pass for the whole warp
// whenever a single lane improves; queueing lets the lanes share that cost.
// The merge applies the exact test against the live list in candidate
// order, so the result is the same as inserting at once.  Four candidates
// are keyed per step with packed .f32x2 arithmetic (the same per-operation
// rounding as the scalar key), and the warp skips the queue code unless one
// of its lanes has a hit among them.
constexpr int KNN_QL = 8;  // queue capacity
constexpr int KNN_U = 4;   // candidates per step (KNN_TILE is a multiple)

__device__ __forceinline__ u64 knn_key2(u64 qx, u64 qy, u64 qz, u64 cx, u64 cy, u64 cz) {
  const u64 dx = sub2(qx, cx), dy = sub2(qy, cy), dz = sub2(qz, cz);
  return add2(add2(mul2(dx, dx), mul2(dy, dy)), mul2(dz, dz));
}

// Scan candidates P[base .. base + n) in index order for one query q held by
// this thread; tile staging is shared by the block (all threads of the block
// must call this with the same base and n, so the warp votes are uniform).
// The tile is stored as three coordinate arrays.  Indices written are global.
template <int KC>
__device__ __forceinline__ void knn_scan(const float4* __restrict__ P, int64_t base, int n, float4 q, float* kd,
                                         int* ki, float* tile, float* qks, int* qis) {
  float* tx = tile;
  float* ty = tile + KNN_TILE;
  float* tz = tile + 2 * KNN_TILE;
#pragma unroll
  for (int m = 0; m < KC; ++m) {
    kd[m] = INFINITY;
    ki[m] = INT_MAX;
  }
  // this thread's queue: slot s at [s * KNN_TPB + threadIdx.x] (conflict-free)
  float* qk = qks + threadIdx.x;
  int* qi = qis + threadIdx.x;
  int qn = 0;
  float thr = INFINITY;
  const u64 qx = pk2(q.x, q.x), qy = pk2(q.y, q.y), qz = pk2(q.z, q.z);
  for (int t0 = 0; t0 < n; t0 += KNN_TILE) {
    const int cnt = min(KNN_TILE, n - t0);
    __syncthreads();
    for (int t = threadIdx.x; t < cnt; t += KNN_TPB) {
      const float4 c = P[base + t0 + t];
      tx[t] = c.x;
      ty[t] = c.y;
      tz[t] = c.z;
    }
    __syncthreads();
    const int idx0 = (int)(base + t0);
    int jj = 0;
    if (KC == 1) {
      for (; jj < cnt; ++jj) knn_insert<KC>(knn_key(q, make_float4(tx[jj], ty[jj], tz[jj], 0.f)), idx0 + jj, kd, ki);
      continue;
    }
    for (; jj + KNN_U <= cnt; jj += KNN_U) {
      const ulonglong2 X = *reinterpret_cast<const ulonglong2*>(tx + jj);
      const ulonglong2 Y = *reinterpret_cast<const ulonglong2*>(ty + jj);
      const ulonglong2 Z = *reinterpret_cast<const ulonglong2*>(tz + jj);
      float key[KNN_U];
      upk2(knn_key2(qx, qy, qz, X.x, Y.x, Z.x), key[0], key[1]);
      upk2(knn_key2(qx, qy, qz, X.y, Y.y, Z.y), key[2], key[3]);
      const bool hit = (key[0] < thr) | (key[1] < thr) | (key[2] < thr) | (key[3] < thr);
      if (__any_sync(0xffffffffu, hit)) {
#pragma unroll
        for (int u = 0; u < KNN_U; ++u) {
          if (key[u] < thr) {
            qk[qn * KNN_TPB] = key[u];
            qi[qn * KNN_TPB] = idx0 + jj + u;
            ++qn;
          }
        }
        if (__any_sync(0xffffffffu, qn > KNN_QL - KNN_U)) {
          for (int sl = 0; sl < qn; ++sl) knn_insert<KC>(qk[sl * KNN_TPB], qi[sl * KNN_TPB], kd, ki);
          qn = 0;
          thr = kd[KC - 1];
        }
      }
    }
    if (jj < cnt) {  // ragged end of the last tile: empty the queue, then insert directly
      for (int sl = 0; sl < qn; ++sl) knn_insert<KC>(qk[sl * KNN_TPB], qi[sl * KNN_TPB], kd, ki);
      qn = 0;
      for (; jj < cnt; ++jj) knn_insert<KC>(knn_key(q, make_float4(tx[jj], ty[jj], tz[jj], 0.f)), idx0 + jj, kd, ki);
      thr = kd[KC - 1];
    }
  }
  for (int sl = 0; sl < qn; ++sl) knn_insert<KC>(qk[sl * KNN_TPB], qi[sl * KNN_TPB], kd, ki);
}

template <int KC>
__global__ void __launch_bounds__(KNN_TPB, KC > 16 ? 2 : 4) knn_brute_kernel(const float4* __restrict__ P, int n,
                                                            int k, int32_t* __restrict__ out) {
  __shared__ __align__(16) float tile[3 * KNN_TILE];
  __shared__ float qks[KNN_QL * KNN_TPB];
  __shared__ int qis[KNN_QL * KNN_TPB];
  const int qi = blockIdx.x * KNN_TPB + threadIdx.x;
  const float4 q = P[qi < n ? qi : n - 1];
  float kd[KC];
  int ki[KC];
  knn_scan<KC>(P, 0, n, q, kd, ki, tile, qks, qis);
  if (qi < n) {
#pragma unroll
    for (int m = 0; m < KC; ++m)
      if (m < k) out[(int64_t)qi * k + m] = ki[m];
  }
}

// Many clouds in one launch: block b handles queries [q0, q0 + KNN_TPB) of
// cloud c = table[b].x (q0 = table[b].y), each against its own cloud only.
template <int KC>
__global__ void __launch_bounds__(KNN_TPB, KC > 16 ? 2 : 4) knn_brute_multi_kernel(const float4* __restrict__ P,
                                                                  const int64_t* __restrict__ off,
                                                                  const int2* __restrict__ table, int k,
                                                                  int32_t* __restrict__ out) {
  __shared__ __align__(16) float tile[3 * KNN_TILE];
  __shared__ float qks[KNN_QL * KNN_TPB];
  __shared__ int qis[KNN_QL * KNN_TPB];
  const int2 e = table[blockIdx.x];
  const int64_t base = off[e.x];
  const int n = (int)(off[e.x + 1] - base);
  const int ql = e.y + threadIdx.x;
  const float4 q = P[base + (ql < n ? ql : n - 1)];
  float kd[KC];
  int ki[KC];
  knn_scan<KC>(P, base, n, q, kd, ki, tile, qks, qis);
  if (ql < n) {
#pragma unroll
    for (int m = 0; m < KC; ++m)
      if (m < k) out[(base + ql) * k + m] = ki[m];
  }
}

// Nearest reference point of arbitrary query points (change detection):
// the same exact key and (key, index) order as the kNN, k = 1.
__global__ void __launch_bounds__(KNN_TPB) nearest_kernel(const float4* __restrict__ P, int n,
                                                          const float* __restrict__ q3, int nq,
                                                          int32_t* __restrict__ idx_out, float* __restrict__ key_out) {
  __shared__ __align__(16) float tile[3 * KNN_TILE];
  const int qi = blockIdx.x * KNN_TPB + threadIdx.x;
  const int qc = qi < nq ? qi : nq - 1;
  const float4 q = make_float4(q3[3 * (size_t)qc], q3[3 * (size_t)qc + 1], q3[3 * (size_t)qc + 2], 0.f);
  float kd[1];
  int ki[1];
  knn_scan<1>(P, 0, n, q, kd, ki, tile, nullptr, nullptr);
  if (qi < nq) {
    if (idx_out) idx_out[qi] = ki[0];
    if (key_out) key_out[qi] = kd[0];
  }
}

cudaError_t launch_nearest(Launch L, const float4* P, int n, const float* q3, int nq, int32_t* idx_out,
                           float* key_out) {
  if (nq <= 0) return cudaSuccess;
  nearest_kernel<<<(nq + KNN_TPB - 1) / KNN_TPB, KNN_TPB, 0, L.stream>>>(P, n, q3, nq, idx_out, key_out);
  return after_launch(L);
}

__global__ void threshold_kernel(const float* __restrict__ key, int nq, float thr2, uint8_t* __restrict__ mask,
                                 float* __restrict__ dist) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nq) return;
  const float k = key[i];
  mask[i] = k > thr2 ? 1 : 0;
  if (dist) dist[i] = sqrtf(k);
}

cudaError_t launch_threshold(Launch L, const float* key, int nq, float thr2, uint8_t* mask, float* dist) {
  if (nq <= 0) return cudaSuccess;
  threshold_kernel<<<(nq + 255) / 256, 256, 0, L.stream>>>(key, nq, thr2, mask, dist);
  return after_launch(L);
}

cudaError_t launch_knn_multi(Launch L, const float4* P, const int64_t* off_dev, const int2* table_dev,
                             int nblocks, int k, int32_t* out) {
  if (nblocks <= 0) return cudaSuccess;
  if (k <= 8) knn_brute_multi_kernel<8><<<nblocks, KNN_TPB, 0, L.stream>>>(P, off_dev, table_dev, k, out);
  else if (k <= 16) knn_brute_multi_kernel<16><<<nblocks, KNN_TPB, 0, L.stream>>>(P, off_dev, table_dev, k, out);
  else knn_brute_multi_kernel<32><<<nblocks, KNN_TPB, 0, L.stream>>>(P, off_dev, table_dev, k, out);
  return after_launch(L);
}

cudaError_t launch_knn(Launch L, const float4* P, int n, int k, int32_t* out) {
  const unsigned grid = (unsigned)((n + KNN_TPB - 1) / KNN_TPB);
  if (k <= 8) knn_brute_kernel<8><<<grid, KNN_TPB, 0, L.stream>>>(P, n, k, out);
  else if (k <= 16) knn_brute_kernel<16><<<grid, KNN_TPB, 0, L.stream>>>(P, n, k, out);
  else knn_brute_kernel<32><<<grid, KNN_TPB, 0, L.stream>>>(P, n, k, out);
  return after_launch(L);
}

// ---- curvature ----------------------------------------------------------
// a = lambda_min / (lambda_1 + lambda_2 + lambda_3) of the 1/k covariance of
// the k neighbours (float64); lambda_min clamped at 0; 0 for a zero trace.
__global__ void curvature_kernel(const float4* __restrict__ P, const int32_t* __restrict__ nbr,
                                 int n, int k, double* __restrict__ a64, float* __restrict__ a32) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int32_t* nb = nbr + (int64_t)i * k;
  double mx = 0, my = 0, mz = 0;
  for (int m = 0; m < k; ++m) {
    const float4 c = P[nb[m]];
    mx += c.x;
    my += c.y;
    mz += c.z;
  }
  mx /= k;
  my /= k;
  mz /= k;
  double C[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
  for (int m = 0; m < k; ++m) {
    const float4 c = P[nb[m]];
    const double dx = c.x - mx, dy = c.y - my, dz = c.z - mz;
    C[0] += dx * dx; C[1] += dx * dy; C[2] += dx * dz;
    C[4] += dy * dy; C[5] += dy * dz; C[8] += dz * dz;
  }
  C[0] /= k; C[1] /= k; C[2] /= k; C[4] /= k; C[5] /= k; C[8] /= k;
  C[3] = C[1]; C[6] = C[2]; C[7] = C[5];
  const double lmin = sym3_min_eigenvalue(C);
  const double tr = C[0] + C[4] + C[8];
  const double a = tr > 0.0 ? fmax(lmin, 0.0) / tr : 0.0;
  a64[i] = a;
  a32[i] = (float)a;
}

cudaError_t launch_curvature(Launch L, const float4* P, const int32_t* nbr, int n, int k,
                             double* a64, float* a32) {
  const int tpb = 128;
  curvature_kernel<<<(n + tpb - 1) / tpb, tpb, 0, L.stream>>>(P, nbr, n, k, a64, a32);
  return after_launch(L);
}

// ---- radius neighbourhood curvature (Sec. IV) ----------------------------
// The neighbourhood of p is every point q of the cloud (p included) whose
// float32 key (dx*dx + dy*dy) + dz*dz, each operation rounded on its own,
// is <= float32(scale^2 * e), e the largest eigenvalue of the cloud's 1/n
// covariance (radius sqrt(e), Sec. IV).  Its 1/|N| covariance gives
// a = lambda_min / trace.  Two passes over the cloud: the first finds the
// neighbourhood's mean c (offsets summed in float32 per tile, float64
// across tiles); the second accumulates the centred moments
// sum (q - p - c) and sum (q - p - c)(q - p - c)^T in float64, so that a
// near-planar neighbourhood keeps its small eigenvalue.
constexpr int RAD_TPB = 128;
constexpr int RAD_TILE = 512;

__device__ __forceinline__ bool radius_member(float4 q, float4 c, float r2, float& dx, float& dy, float& dz) {
  dx = __fsub_rn(c.x, q.x);
  dy = __fsub_rn(c.y, q.y);
  dz = __fsub_rn(c.z, q.z);
  const float key = __fadd_rn(__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)), __fmul_rn(dz, dz));
  return key <= r2;
}

__global__ void __launch_bounds__(RAD_TPB)
    radius_curvature_kernel(const float4* __restrict__ P, int n, const double* __restrict__ e_dev, double scale2,
                            double* __restrict__ a64, float* __restrict__ a32, int* __restrict__ count_out) {
  __shared__ float4 tile[RAD_TILE];
  const int i = blockIdx.x * RAD_TPB + threadIdx.x;
  const float4 q = P[i < n ? i : n - 1];
  const float r2 = (float)(scale2 * e_dev[0]);
  // pass 1: count and mean offset
  double M[3] = {0, 0, 0};
  int cnt = 0;
  for (int base = 0; base < n; base += RAD_TILE) {
    const int m = min(RAD_TILE, n - base);
    __syncthreads();
    for (int t = threadIdx.x; t < m; t += RAD_TPB) tile[t] = P[base + t];
    __syncthreads();
    float s[3] = {0, 0, 0};
    for (int jj = 0; jj < m; ++jj) {
      float dx, dy, dz;
      if (radius_member(q, tile[jj], r2, dx, dy, dz)) {
        ++cnt;
        s[0] += dx; s[1] += dy; s[2] += dz;
      }
    }
    M[0] += s[0]; M[1] += s[1]; M[2] += s[2];
  }
  const double k = (double)cnt;
  const double c[3] = {M[0] / k, M[1] / k, M[2] / k};
  // pass 2: centred first and second moments in float64
  double S[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
  for (int base = 0; base < n; base += RAD_TILE) {
    const int m = min(RAD_TILE, n - base);
    __syncthreads();
    for (int t = threadIdx.x; t < m; t += RAD_TPB) tile[t] = P[base + t];
    __syncthreads();
    for (int jj = 0; jj < m; ++jj) {
      float dx, dy, dz;
      if (radius_member(q, tile[jj], r2, dx, dy, dz)) {
        const double ex = (double)dx - c[0], ey = (double)dy - c[1], ez = (double)dz - c[2];
        S[0] += ex; S[1] += ey; S[2] += ez;
        S[3] += ex * ex; S[4] += ex * ey; S[5] += ex * ez;
        S[6] += ey * ey; S[7] += ey * ez; S[8] += ez * ez;
      }
    }
  }
  if (i >= n) return;
  const double mx = S[0] / k, my = S[1] / k, mz = S[2] / k;
  double C[9];
  C[0] = S[3] / k - mx * mx; C[1] = S[4] / k - mx * my; C[2] = S[5] / k - mx * mz;
  C[4] = S[6] / k - my * my; C[5] = S[7] / k - my * mz; C[8] = S[8] / k - mz * mz;
  C[3] = C[1]; C[6] = C[2]; C[7] = C[5];
  const double lmin = sym3_min_eigenvalue(C);
  const double tr = C[0] + C[4] + C[8];
  const double a = tr > 0.0 ? fmax(lmin, 0.0) / tr : 0.0;
  a64[i] = a;
  a32[i] = (float)a;
  if (count_out) count_out[i] = cnt;
}

cudaError_t launch_radius_curvature(Launch L, const float4* P, int n, const double* e_dev, double scale2,
                                    double* a64, float* a32, int* count_out) {
  radius_curvature_kernel<<<(n + RAD_TPB - 1) / RAD_TPB, RAD_TPB, 0, L.stream>>>(P, n, e_dev, scale2, a64, a32,
                                                                                 count_out);
  return after_launch(L);
}

// ---- fixed-order float64 reductions ------------------------------------
// Pass 1: per-block sums of an NV-vector per point (fixed grid, fixed order).
struct SumXYZ {
  const float4* P;
  __device__ void operator()(int64_t i, double (&v)[3]) const {
    const float4 c = P[i];
    v[0] += c.x; v[1] += c.y; v[2] += c.z;
  }
};
struct ScatterXYZ {
  const float4* P;
  const double* mean;
  __device__ void operator()(int64_t i, double (&v)[6]) const {
    const float4 c = P[i];
    const double dx = c.x - mean[0], dy = c.y - mean[1], dz = c.z - mean[2];
    v[0] += dx * dx; v[1] += dx * dy; v[2] += dx * dz;
    v[3] += dy * dy; v[4] += dy * dz; v[5] += dz * dz;
  }
};
struct SumA {
  const double* a;
  __device__ void operator()(int64_t i, double (&v)[1]) const { v[0] += a[i]; }
};
struct VarA {
  const double* a;
  const double* mean_sum;  // sum of a; mean = sum / n
  double inv_n;
  __device__ void operator()(int64_t i, double (&v)[1]) const {
    const double d = a[i] - mean_sum[0] * inv_n;
    v[0] += d * d;
  }
};

template <int NV, class Fn>
__global__ void __launch_bounds__(RED_THREADS) reduce_pass_kernel(int64_t n, Fn fn, double* part) {
  __shared__ double sh[NV][RED_THREADS];
  double v[NV];
#pragma unroll
  for (int q = 0; q < NV; ++q) v[q] = 0.0;
  const int64_t stride = (int64_t)gridDim.x * RED_THREADS;
  for (int64_t i = blockIdx.x * (int64_t)RED_THREADS + threadIdx.x; i < n; i += stride) fn(i, v);
  block_sum<NV>(v, sh);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int q = 0; q < NV; ++q) part[blockIdx.x * NV + q] = v[q];
  }
}

// Pass 2: one block sums the per-block partials in fixed order into out[NV].
template <int NV>
__global__ void __launch_bounds__(RED_THREADS) reduce_final_kernel(const double* part, int nb,
                                                                   double* out) {
  __shared__ double sh[NV][RED_THREADS];
  double v[NV];
#pragma unroll
  for (int q = 0; q < NV; ++q) v[q] = 0.0;
  for (int b = threadIdx.x; b < nb; b += RED_THREADS) {
#pragma unroll
    for (int q = 0; q < NV; ++q) v[q] += part[b * NV + q];
  }
  block_sum<NV>(v, sh);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int q = 0; q < NV; ++q) out[q] = v[q];
  }
}

__global__ void mean_from_sum_kernel(double* mean, int64_t n) {
  if (threadIdx.x == 0) {
    mean[0] /= (double)n;
    mean[1] /= (double)n;
    mean[2] /= (double)n;
  }
}

__global__ void scatter_finish_kernel(const double* s6, int64_t n, double* scatter, double* lmax) {
  if (threadIdx.x != 0) return;
  double S[9] = {s6[0], s6[1], s6[2], s6[1], s6[3], s6[4], s6[2], s6[4], s6[5]};
  for (int q = 0; q < 9; ++q) scatter[q] = S[q];
  double C[9];
  for (int q = 0; q < 9; ++q) C[q] = S[q] / (double)n;
  double lam[3];
  sym3_eigenvalues(C, lam);
  *lmax = lam[2];
}

cudaError_t launch_cloud_stats(Launch L, const float4* P, int n, double* part, double* mean,
                               double* scatter, double* lmax) {
  const int nb = red_blocks(n);
  reduce_pass_kernel<3, SumXYZ><<<nb, RED_THREADS, 0, L.stream>>>(n, SumXYZ{P}, part);
  reduce_final_kernel<3><<<1, RED_THREADS, 0, L.stream>>>(part, nb, mean);
  mean_from_sum_kernel<<<1, 32, 0, L.stream>>>(mean, n);
  // the 6 scatter sums go to part + RED_MAX_BLOCKS*6 .. as the final output slot
  double* s6 = part + (size_t)RED_MAX_BLOCKS * 6;
  reduce_pass_kernel<6, ScatterXYZ><<<nb, RED_THREADS, 0, L.stream>>>(n, ScatterXYZ{P, mean}, part);
  reduce_final_kernel<6><<<1, RED_THREADS, 0, L.stream>>>(part, nb, s6);
  scatter_finish_kernel<<<1, 32, 0, L.stream>>>(s6, n, scatter, lmax);
  if (L.counter) *L.counter += 6;
  return cudaGetLastError();
}

__global__ void sigma_finish_kernel(const double* sums, int64_t n, double sigma_user,
                                    double* sigma_out, double* asum_out) {
  if (threadIdx.x != 0) return;
  if (asum_out) *asum_out = sums[0];
  if (sigma_user > 0.0) {
    *sigma_out = sigma_user;
    return;
  }
  const double sd = sqrt(sums[1] / (double)n);
  *sigma_out = sd >= 1e-12 ? sd : 1.0;
}

cudaError_t launch_sigma(Launch L, const double* a64, int n, double sigma_user, double* part,
                         double* sigma_out, double* asum_out) {
  const int nb = red_blocks(n);
  double* sums = part + (size_t)RED_MAX_BLOCKS * 6 + 8;  // [0]: sum a, [1]: sum (a - mean)^2
  reduce_pass_kernel<1, SumA><<<nb, RED_THREADS, 0, L.stream>>>(n, SumA{a64}, part);
  reduce_final_kernel<1><<<1, RED_THREADS, 0, L.stream>>>(part, nb, sums);
  reduce_pass_kernel<1, VarA><<<nb, RED_THREADS, 0, L.stream>>>(n, VarA{a64, sums, 1.0 / n}, part);
  reduce_final_kernel<1><<<1, RED_THREADS, 0, L.stream>>>(part, nb, sums + 1);
  sigma_finish_kernel<<<1, 32, 0, L.stream>>>(sums, n, sigma_user, sigma_out, asum_out);
  if (L.counter) *L.counter += 5;
  return cudaGetLastError();
}

__global__ void scale_double_kernel(double* v, double f) {
  if (threadIdx.x == 0 && blockIdx.x == 0) *v *= f;
}

cudaError_t launch_scale_double(Launch L, double* v, double f) {
  scale_double_kernel<<<1, 32, 0, L.stream>>>(v, f);
  return after_launch(L);
}

// ---- caller-supplied curvature --------------------------------------------
__global__ void check_curvature_kernel(const double* __restrict__ a64, int n, float* __restrict__ a32,
                                       int* __restrict__ err) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double a = a64[i];
  if (!(a >= 0.0 && a <= 1.0)) atomicOr(err, ERR_NONFINITE);
  a32[i] = (float)a;
}

cudaError_t launch_check_curvature(Launch L, const double* a64, int n, float* a32, int* err) {
  check_curvature_kernel<<<(n + 255) / 256, 256, 0, L.stream>>>(a64, n, a32, err);
  return after_launch(L);
}

// ---- force-kernel records ----------------------------------------------
// s_ij = exp(-(aX - aY)^2 / sigma^2) = 2^(-(a_hat_X - a_hat_Y)^2) with
// a_hat = a * sqrt(log2 e) / sigma (Eq. 3).  In the mode g = aX aY s (Eq. 10)
// the factor aX enters the exponent as L = log2 aX (stored negated, -L >= 0)
// and aY multiplies the per-point sums; in the mode g = s, L = 0 and the aY
// factor is 1.  Reference coordinates are shifted by the reference mean so
// that |X'|^2 + |Y'|^2 - 2 X'.Y' loses little to cancellation.  The records
// are written tile-major as structure-of-arrays (FORCE_TJ points per tile).
// Padding records carry -L = +inf, so their weight is exactly 0.
__device__ __forceinline__ void write_x_record(int i, int n, const float4* __restrict__ X4,
                                               const double* __restrict__ aX64, int g_mode, const DevStats& st,
                                               float* __restrict__ Xr, float* __restrict__ XA) {
  const double kscale = sqrt(1.4426950408889634) / st.sigma;  // sqrt(log2 e) / sigma
  const size_t t = (size_t)(i / FORCE_TJ), r = (size_t)(i % FORCE_TJ);
  float* xr = Xr + t * 4 * FORCE_TJ + r;
  float* xa = XA + t * 2 * FORCE_TJ + r;
  if (i < n) {
    const float4 c = X4[i];
    const float x = (float)((double)c.x - st.xbar[0]);
    const float y = (float)((double)c.y - st.xbar[1]);
    const float z = (float)((double)c.z - st.xbar[2]);
    const double nn = (double)x * x + (double)y * y + (double)z * z;
    xr[0] = x;
    xr[FORCE_TJ] = y;
    xr[2 * FORCE_TJ] = z;
    xr[3 * FORCE_TJ] = (float)nn;
    const double a = aX64[i];
    const float nL = g_mode == 1 ? (a > 0.0 ? (float)(-log2(a)) : INFINITY) : 0.f;
    xa[0] = (float)(a * kscale);
    xa[FORCE_TJ] = nL;
  } else {
    xr[0] = xr[FORCE_TJ] = xr[2 * FORCE_TJ] = xr[3 * FORCE_TJ] = 0.f;
    xa[0] = 0.f;
    xa[FORCE_TJ] = INFINITY;
  }
}

__device__ __forceinline__ void write_y_record(int i, int m, const float4* __restrict__ Y4,
                                               const double* __restrict__ aY64, const DevStats& st,
                                               float4* __restrict__ Y0r) {
  if (i < m) {
    const double kscale = sqrt(1.4426950408889634) / st.sigma;
    const float4 c = Y4[i];
    Y0r[i] = make_float4(c.x, c.y, c.z, (float)(aY64[i] * kscale));
  } else {
    Y0r[i] = make_float4(0.f, 0.f, 0.f, 0.f);
  }
}

__global__ void records_kernel(const float4* __restrict__ X4, const double* __restrict__ aX64,
                               int n, int npad, const float4* __restrict__ Y4,
                               const double* __restrict__ aY64, int m, int mpad, int g_mode,
                               const DevStats* __restrict__ st, float* __restrict__ Xr,
                               float* __restrict__ XA, float4* __restrict__ Y0r) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < npad) write_x_record(i, n, X4, aX64, g_mode, *st, Xr, XA);
  if (i < mpad) write_y_record(i, m, Y4, aY64, *st, Y0r);
}

// Batched records: block (p, part) writes pair p's padded reference tiles and
// template slots (grid-strided over `part`).
__global__ void records_multi_kernel(const float4* __restrict__ X4, const double* __restrict__ aX64,
                                     const float4* __restrict__ Y4, const double* __restrict__ aY64,
                                     const BatchPair* __restrict__ pairs, int g_mode,
                                     const DevStats* __restrict__ st, float* __restrict__ Xr,
                                     float* __restrict__ XA, float4* __restrict__ Y0r) {
  const BatchPair bp = pairs[blockIdx.x];
  const DevStats& S = st[blockIdx.x];
  const int stride = blockDim.x * gridDim.y;
  const int npad = bp.ntiles * FORCE_TJ;
  for (int i = blockIdx.y * blockDim.x + threadIdx.x; i < npad; i += stride)
    write_x_record(i, (int)bp.n, X4 + bp.x0, aX64 + bp.x0, g_mode, S, Xr + (size_t)bp.xtile0 * 4 * FORCE_TJ,
                   XA + (size_t)bp.xtile0 * 2 * FORCE_TJ);
  for (int i = blockIdx.y * blockDim.x + threadIdx.x; i < bp.mpad; i += stride)
    write_y_record(i, (int)bp.m, Y4 + bp.y0, aY64 + bp.y0, S, Y0r + bp.ybase);
}

cudaError_t launch_records_multi(Launch L, const float4* X4, const double* aX64, const float4* Y4,
                                 const double* aY64, const BatchPair* pairs, int npairs, int g_mode,
                                 const DevStats* stats, float4* Xr, float2* XA, float4* Y0r) {
  records_multi_kernel<<<dim3(npairs, 8), 256, 0, L.stream>>>(X4, aX64, Y4, aY64, pairs, g_mode, stats,
                                                               reinterpret_cast<float*>(Xr),
                                                               reinterpret_cast<float*>(XA), Y0r);
  return after_launch(L);
}

// Batched statistics: block p computes, in a fixed order, the reference and
// template means, scatters and largest eigenvalues of pair p, and sigma
// (population std of its reference curvatures, or sigma_user if > 0).
__global__ void __launch_bounds__(RED_THREADS)
    stats_multi_kernel(const float4* __restrict__ X4, const float4* __restrict__ Y4,
                       const double* __restrict__ aX64, const BatchPair* __restrict__ pairs,
                       double sigma_user, DevStats* __restrict__ out) {
  __shared__ double sh[6][RED_THREADS];
  const BatchPair bp = pairs[blockIdx.x];
  DevStats* st = out + blockIdx.x;
  for (int side = 0; side < 2; ++side) {
    const float4* P = side == 0 ? X4 + bp.x0 : Y4 + bp.y0;
    const int64_t n = side == 0 ? bp.n : bp.m;
    double v3[3] = {0, 0, 0};
    for (int64_t i = threadIdx.x; i < n; i += RED_THREADS) {
      const float4 c = P[i];
      v3[0] += c.x; v3[1] += c.y; v3[2] += c.z;
    }
    block_sum<3>(v3, sh);
    const double mean[3] = {v3[0] / n, v3[1] / n, v3[2] / n};
    __syncthreads();
    double v6[6] = {0, 0, 0, 0, 0, 0};
    for (int64_t i = threadIdx.x; i < n; i += RED_THREADS) {
      const float4 c = P[i];
      const double dx = c.x - mean[0], dy = c.y - mean[1], dz = c.z - mean[2];
      v6[0] += dx * dx; v6[1] += dx * dy; v6[2] += dx * dz;
      v6[3] += dy * dy; v6[4] += dy * dz; v6[5] += dz * dz;
    }
    block_sum<6>(v6, sh);
    if (threadIdx.x == 0) {
      const double S[9] = {v6[0], v6[1], v6[2], v6[1], v6[3], v6[4], v6[2], v6[4], v6[5]};
      double C[9], lam[3];
      for (int q = 0; q < 9; ++q) C[q] = S[q] / (double)n;
      sym3_eigenvalues(C, lam);
      double* mo = side == 0 ? st->xbar : st->ybar0;
      double* so = side == 0 ? st->CX : st->S0;
      for (int q = 0; q < 3; ++q) mo[q] = mean[q];
      for (int q = 0; q < 9; ++q) so[q] = S[q];
      if (side == 0) st->eX = lam[2];
      else st->eY0 = lam[2];
    }
    __syncthreads();
  }
  double v1[1] = {0};
  for (int64_t i = threadIdx.x; i < bp.n; i += RED_THREADS) v1[0] += aX64[bp.x0 + i];
  block_sum<1>(v1, sh);
  const double amean = v1[0] / bp.n;
  const double asum = v1[0];
  __syncthreads();
  double v2[1] = {0};
  for (int64_t i = threadIdx.x; i < bp.n; i += RED_THREADS) {
    const double d = aX64[bp.x0 + i] - amean;
    v2[0] += d * d;
  }
  block_sum<1>(v2, sh);
  if (threadIdx.x == 0) {
    st->asum[0] = asum;
    if (sigma_user > 0.0) st->sigma = sigma_user;
    else {
      const double sd = sqrt(v2[0] / bp.n);
      st->sigma = sd >= 1e-12 ? sd : 1.0;
    }
  }
}

cudaError_t launch_stats_multi(Launch L, const float4* X4, const float4* Y4, const double* aX64,
                               const BatchPair* pairs, int npairs, double sigma_user, DevStats* out) {
  stats_multi_kernel<<<npairs, RED_THREADS, 0, L.stream>>>(X4, Y4, aX64, pairs, sigma_user, out);
  return after_launch(L);
}

cudaError_t launch_records(Launch L, const float4* X4, const double* aX64, int n, int npad,
                           const float4* Y4, const double* aY64, int m, int mpad, int g_mode,
                           const DevStats* stats, float4* Xr, float2* XA, float4* Y0r) {
  const int tpb = 256;
  const int tot = npad > mpad ? npad : mpad;
  records_kernel<<<(tot + tpb - 1) / tpb, tpb, 0, L.stream>>>(
      X4, aX64, n, npad, Y4, aY64, m, mpad, g_mode, stats, reinterpret_cast<float*>(Xr),
      reinterpret_cast<float*>(XA), Y0r);
  return after_launch(L);
}

}  // namespace scgr
