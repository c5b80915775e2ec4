// Per-template-point pieces shared by the force, combine and fused
// combine-finalize kernels (included by force.cu and pose.cu; the library is
// built without relocatable device code, so shared device code lives here).
#pragma once
#include "common.cuh"

namespace scgr {

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

// The pose's float32 map (A, b) and the template mean in the centred frame
// as a float pair (ch + cl), all stored with the pose (no float64 work per
// thread).
struct PointFrame {
  float A[9], b[3], ch[3], cl[3];
  __device__ __forceinline__ explicit PointFrame(const DevPose* ps) {
#pragma unroll
    for (int q = 0; q < 9; ++q) A[q] = ps->A[q];
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      b[q] = ps->b[q];
      ch[q] = ps->ych[q];
      cl[q] = ps->ycl[q];
    }
  }
};

// Force on template slot i from its S split partials (sum_j w X', sum_j w)
// at stride pstride: the splits added in order with Kahan compensation, then
// f = aY (S - Y' W) from an exact product and an exact two-sum, so f is as
// accurate as float allows even when S and Y' W nearly cancel; W_i = aY W.
// Returns (f, W_i).
__device__ __forceinline__ float4 point_fw(const float4* __restrict__ pbase, size_t pstride, int S, int i,
                                           const float4 y0, float ay, const PointFrame& fr) {
  float Wh = 0.f, Wc = 0.f, Sh[3] = {0.f, 0.f, 0.f}, Sc[3] = {0.f, 0.f, 0.f};
  // splits in order, eight loads in flight per step (small templates leave
  // few threads per SM, so the pass over the splits is load-latency bound)
  for (int s = 0; s < S; s += 8) {
    float4 pp[8];
#pragma unroll
    for (int u = 0; u < 8; ++u)
      if (s + u < S) pp[u] = pbase[(size_t)(s + u) * pstride + i];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      if (s + u < S) {
        kahan_add(Wh, Wc, pp[u].x);
        kahan_add(Sh[0], Sc[0], pp[u].y);
        kahan_add(Sh[1], Sc[1], pp[u].z);
        kahan_add(Sh[2], Sc[2], pp[u].w);
      }
    }
  }
  float y[3];
  template_point(y0, fr.A, fr.b, y[0], y[1], y[2]);
  float f[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    // D = (Sh - Sc) - y (Wh - Wc): y Wh = p + pe exactly, Sh - p = dh + dl
    // exactly.  Each step is an explicitly rounded operation, so the
    // compiler cannot contract y Wh into the subtraction (the error-free
    // transformations need p and dh rounded on their own).
    const float p = __fmul_rn(y[a], Wh);
    const float pe = __fmaf_rn(y[a], Wh, -p);
    const float dh = __fsub_rn(Sh[a], p);
    const float bv = __fsub_rn(dh, Sh[a]);
    const float dl = __fadd_rn(__fsub_rn(Sh[a], __fsub_rn(dh, bv)), __fsub_rn(-p, bv));
    const float D = __fadd_rn(dh, __fadd_rn(__fsub_rn(dl, pe), __fmaf_rn(y[a], Wc, -Sc[a])));
    f[a] = ay * D;
  }
  return make_float4(f[0], f[1], f[2], ay * (Wh - Wc));
}

// Adds a point's f, W_i and f (x) (Y' - ybar') to acc[13] (fw = point_fw's
// result for the template record y0).  The additions are explicitly rounded,
// so the compiler cannot fuse point_fw's last products into them where both
// are inlined together: every kernel adds the same rounded per-point terms,
// whether fw comes straight from point_fw or through shared memory.
__device__ __forceinline__ void point_acc(const float4 fw, const float4 y0, const PointFrame& fr, float (&acc)[13]) {
  float y[3];
  template_point(y0, fr.A, fr.b, y[0], y[1], y[2]);
  const float f[3] = {fw.x, fw.y, fw.z};
  float c[3];
#pragma unroll
  for (int q = 0; q < 3; ++q) c[q] = (y[q] - fr.ch[q]) - fr.cl[q];
  acc[0] = __fadd_rn(acc[0], f[0]);
  acc[1] = __fadd_rn(acc[1], f[1]);
  acc[2] = __fadd_rn(acc[2], f[2]);
  acc[3] = __fadd_rn(acc[3], fw.w);
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int bb = 0; bb < 3; ++bb) acc[4 + 3 * a + bb] = fmaf(f[a], c[bb], acc[4 + 3 * a + bb]);
}

// point_fw then point_acc; optionally stores (f, W_i) to f4out[i].
__device__ __forceinline__ void point_force(const float4* __restrict__ pbase, size_t pstride, int S, int i,
                                            const float4 y0, float ay, const PointFrame& fr, float (&acc)[13],
                                            float4* __restrict__ f4out) {
  const float4 fw = point_fw(pbase, pstride, S, i, y0, ay, fr);
  point_acc(fw, y0, fr, acc);
  if (f4out) f4out[i] = fw;
}

// Reduce 16 doubles over a warp by recursive halving: lane L ends with the
// warp total of quantity 8 b4 + 4 b3 + 2 b2 + b1 (b_k = bit k of L), 16
// additions per lane instead of 80 for a butterfly per quantity.
__device__ __forceinline__ void warp_reduce16(double (&v)[16]) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int lvl = 0; lvl < 4; ++lvl) {
    const int off = 16 >> lvl;
    const int half = 8 >> lvl;
    const bool upper = (lane & off) != 0;
#pragma unroll
    for (int q = 0; q < half; ++q) {
      const double send = upper ? v[q] : v[q + half];
      const double keep = upper ? v[q + half] : v[q];
      v[q] = keep + __shfl_xor_sync(0xffffffffu, send, off);
    }
  }
  v[0] += __shfl_xor_sync(0xffffffffu, v[0], 1);
}

// Quantity index that lane `lane` holds after warp_reduce16 (valid on even lanes).
__device__ __forceinline__ int warp_reduce16_slot(int lane) {
  return ((lane >> 4) & 1) * 8 + ((lane >> 3) & 1) * 4 + ((lane >> 2) & 1) * 2 + ((lane >> 1) & 1);
}

}  // namespace scgr
