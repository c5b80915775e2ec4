// All-pairs shape-weighted force (Eq. 5 with Eq. 3, Eq. 10, Eq. 11) and its
// reduction to the total force, weight and torque moment (Eq. 5.5, Eq. 6).
//
// For template point Y_i (M of them) and reference point X_j (N of them):
//   w_ij = g(s_ij) d_ij^(p-1),   f_i = -sum_j w_ij (Y_i - X_j),
//   W_i  = sum_j w_ij.
// The kernel accumulates, per template point, sum_j w_ij and sum_j w_ij X_j;
// the combine kernel forms f_i = aY (sum_j w X_j - Y_i sum_j w) afterwards
// from an exact product and an exact two-sum.
//
// Per pair (float32): d^2 = |X'|^2 + |Y'|^2 - 2 X'.Y' (one add, three FMAs),
// the similarity-and-aX factor 2^-(u^2 - L), u = a_hat_X - a_hat_Y (one sub,
// one FMA, one ex2), the distance factor (sqrt for p = 2, folded into the ex2
// exponent through lg2 for general p), and four accumulations.
//
// The FP32 arithmetic runs on packed pairs (Blackwell add/sub/mul/fma
// .f32x2): each instruction handles reference points j and j+1 for one
// template point, so a pair costs 5.5 FP32-pipe issue slots plus its two
// special-function (MUFU) operations, and the MUFU unit becomes the limit.
// Reference tiles are stored tile-major as structure-of-arrays
// (x, y, z, |X'|^2 | a_hat, -L), so a 128-bit shared-memory broadcast delivers
// four consecutive points of one field.
//
// Layout of the work: grid.x covers template points (P per thread, TPB
// threads), grid.y splits the reference range so that the grid has many
// waves on 152 SMs.  Each staged tile's sums are accumulated in plain float32
// (two lanes per point) and then added to the running per-point sums with
// Kahan compensation (kept in registers, or in shared memory for the shape
// that holds 4 points per thread); each split writes its per-point partial
// (float4), and the combine kernel adds the splits per point in a fixed order
// (Kahan) and the points in float64, so results are deterministic.
#include <cmath>

#include "common.cuh"
#include "ex2_poly.cuh"
#include "pointsum.cuh"

namespace scgr {

// 2^-x
__device__ __forceinline__ float ex2_neg(float x) {
  float y;
  asm("{ .reg .f32 t; neg.f32 t, %1; ex2.approx.ftz.f32 %0, t; }" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float lg2_approx(float x) {
  float y;
  asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float rsqrt_approx(float x) {
  float y;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float sqrt_approx(float x) {
  float y;
  asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

constexpr float RSQRT_CAP = 1e18f;

// 2^-e for e >= 0 on the FP32 pipe, both lanes (Cody-Waite reduction):
// e = n + g with n = round(e), g in [-1/2, 1/2]; 2^-g from the degree-5
// minimax polynomial of ex2_poly.cuh (relative error < 2^-22 in float32),
// and 2^-n added to the exponent field.  Adding 1.5 * 2^23 rounds e to an
// integer held in the low mantissa bits: t = 1.5 * 2^23 - n, whose bit
// pattern shifted left by 23 is -n << 23 for |n| < 256.  Results below
// 2^-125.5 (e >= 125.5, including e = +inf) are 0, as the special-function
// unit's flushing ex2 gives below 2^-126.
constexpr float EX2_ROUND = 12582912.0f;  // 1.5 * 2^23
constexpr float EX2_POLY_MAX = 125.5f;
__device__ __forceinline__ u64 ex2_neg_poly2(u64 e) {
  const u64 R2 = pk2(EX2_ROUND, EX2_ROUND);
  const u64 t = sub2(R2, e);   // 1.5 * 2^23 - round(e)
  const u64 nf = sub2(t, R2);  // -round(e), exact
  const u64 g = add2(e, nf);   // e - round(e), exact
  u64 q = fma2(pk2(EX2_POLY_C5, EX2_POLY_C5), g, pk2(EX2_POLY_C4, EX2_POLY_C4));
  q = fma2(q, g, pk2(EX2_POLY_C3, EX2_POLY_C3));
  q = fma2(q, g, pk2(EX2_POLY_C2, EX2_POLY_C2));
  q = fma2(q, g, pk2(EX2_POLY_C1, EX2_POLY_C1));
  q = fma2(q, g, pk2(EX2_POLY_C0, EX2_POLY_C0));
  float t0, t1, q0, q1, e0, e1;
  upk2(t, t0, t1);
  upk2(q, q0, q1);
  upk2(e, e0, e1);
  const float r0 = __uint_as_float(__float_as_uint(q0) + (__float_as_uint(t0) << 23));
  const float r1 = __uint_as_float(__float_as_uint(q1) + (__float_as_uint(t1) << 23));
  return pk2(e0 < EX2_POLY_MAX ? r0 : 0.f, e1 < EX2_POLY_MAX ? r1 : 0.f);
}

// One packed pair update: reference points (j, j+1) against one template point.
// POLY (p = 2 only): the factor 2^-ep on the FP32 pipe instead of the
// special-function unit.
template <int PM, bool POLY = false>
__device__ __forceinline__ void pair2(u64 xv, u64 yv, u64 zv, u64 nv, u64 av, u64 lv, u64 mx, u64 my,
                                      u64 mz, u64 ny, u64 ah, u64 nq, u64& W, u64& Sx, u64& Sy, u64& Sz) {
  u64 d2 = add2(nv, ny);
  d2 = fma2(xv, mx, d2);
  d2 = fma2(yv, my, d2);
  d2 = fma2(zv, mz, d2);
  const u64 u = sub2(av, ah);
  const u64 ep = fma2(u, u, lv);  // u^2 - L >= 0; the weight is 2^-ep times the distance factor
  u64 w;
  if (PM == 1) {
    float e0, e1;
    upk2(ep, e0, e1);
    w = pk2(ex2_neg(e0), ex2_neg(e1));
  } else if (PM == 2) {
    float e0, e1, q0, q1;
    upk2(d2, q0, q1);
    const u64 dd = pk2(sqrt_approx(fabsf(q0)), sqrt_approx(fabsf(q1)));
    if (POLY) {
      w = mul2(ex2_neg_poly2(ep), dd);
    } else {
      upk2(ep, e0, e1);
      w = mul2(pk2(ex2_neg(e0), ex2_neg(e1)), dd);
    }
  } else if (PM == 3) {
    float e0, e1;
    upk2(ep, e0, e1);
    w = mul2(pk2(ex2_neg(e0), ex2_neg(e1)), d2);
  } else if (PM == 4) {
    // p = 2 with d = d^2 / sqrt(|d^2|): a reciprocal square root and one more
    // packed multiply (kept as a tunable alternative: on GB300 rsqrt and sqrt
    // occupy the special-function unit equally, so this form is slower).
    // The cap keeps d^2 = 0 at weight 0 (0 * inf would be NaN); a d^2 below
    // the rounding of its own terms may come out with either sign.
    float e0, e1, q0, q1;
    upk2(ep, e0, e1);
    upk2(d2, q0, q1);
    const u64 r = pk2(fminf(rsqrt_approx(fabsf(q0)), RSQRT_CAP), fminf(rsqrt_approx(fabsf(q1)), RSQRT_CAP));
    w = mul2(mul2(pk2(ex2_neg(e0), ex2_neg(e1)), d2), r);
  } else {
    float q0, q1;
    upk2(d2, q0, q1);
    const u64 t = fma2(nq, pk2(lg2_approx(fabsf(q0)), lg2_approx(fabsf(q1))), ep);  // ep - q log2 d^2
    float t0, t1;
    upk2(t, t0, t1);
    w = pk2(ex2_neg(t0), ex2_neg(t1));
  }
  W = add2(W, w);
  Sx = fma2(w, xv, Sx);
  Sy = fma2(w, yv, Sy);
  Sz = fma2(w, zv, Sz);
}

// Running per-point sums of the force kernel and their Kahan compensations:
// in registers (KS = false) or in shared memory (KS = true, which frees 8
// registers per template point for more pair updates in flight).  The
// shared-memory form keeps value v of point q of thread tid at
// sk[(8 q + v) TPB + tid], so a warp's accesses are consecutive.
template <int P, int TPB, bool KS>
struct RunningSums {
  float h[P][4], c[P][4];
  float* sk;
  __device__ __forceinline__ RunningSums(float* sk_) : sk(sk_) {
#pragma unroll
    for (int q = 0; q < P; ++q)
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        if (KS) {
          sk[(8 * q + v) * TPB + threadIdx.x] = 0.f;
          sk[(8 * q + 4 + v) * TPB + threadIdx.x] = 0.f;
        } else {
          h[q][v] = c[q][v] = 0.f;
        }
      }
  }
  // add the tile sums (two packed lanes each) of point q
  __device__ __forceinline__ void add(int q, u64 w, u64 x, u64 y, u64 z) {
    const u64 in[4] = {w, x, y, z};
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      float l0, l1;
      upk2(in[v], l0, l1);
      if (KS) {
        float* hs = sk + (8 * q + v) * TPB + threadIdx.x;
        float* cs = sk + (8 * q + 4 + v) * TPB + threadIdx.x;
        float hv = *hs, cv = *cs;
        kahan_add(hv, cv, l0 + l1);
        *hs = hv;
        *cs = cv;
      } else {
        kahan_add(h[q][v], c[q][v], l0 + l1);
      }
    }
  }
  __device__ __forceinline__ float4 result(int q) const {
    if (KS) {
      const float* hs = sk + 8 * q * TPB + threadIdx.x;
      return make_float4(hs[0] - hs[4 * TPB], hs[TPB] - hs[5 * TPB], hs[2 * TPB] - hs[6 * TPB],
                         hs[3 * TPB] - hs[7 * TPB]);
    }
    return make_float4(h[q][0] - c[q][0], h[q][1] - c[q][1], h[q][2] - c[q][2], h[q][3] - c[q][3]);
  }
};

// The work of one block: template points [ibase, ibase + P*TPB) of the
// padded record array against reference tiles [t0, t1), at pose *ps; writes
// one float4 partial per template point to outbase[0 .. P*TPB).  SUB record
// tiles of TJ points are staged together (sT holds SUB*TJ points per row);
// a stage past t1 is filled with zero-weight entries (-L = +inf).
// HALF (one tile, SUB = 1): the block takes entries [jlo, jlo + TJ / 2) of
// its tile, half the dependent steps per thread for the smallest problems.
template <int P, int PM, int TPB, int TJ, bool KS, int SUB, int EXO = 0, bool HALF = false>
__device__ __forceinline__ void force_block(float (&sT)[6][TJ * SUB], float* sk, const float* __restrict__ Xr,
                                            const float* __restrict__ XA, int t0, int t1,
                                            const float4* __restrict__ Y0r, int ibase, const DevPose* ps,
                                            float qexp, float4* __restrict__ outbase, int jlo = 0) {
  static_assert(!HALF || SUB == 1, "half tiles stage one tile at a time");
  const int tid = threadIdx.x;
  float A[9], b[3];
#pragma unroll
  for (int q = 0; q < 9; ++q) A[q] = ps->A[q];
#pragma unroll
  for (int q = 0; q < 3; ++q) b[q] = ps->b[q];

  u64 mx[P], my[P], mz[P], ny[P], ah[P];
#pragma unroll
  for (int q = 0; q < P; ++q) {
    const float4 y0 = Y0r[ibase + q * TPB + tid];
    float yx, yy, yz;
    template_point(y0, A, b, yx, yy, yz);
    const float n = fmaf(yz, yz, fmaf(yy, yy, yx * yx));
    mx[q] = pk2(-2.f * yx, -2.f * yx);
    my[q] = pk2(-2.f * yy, -2.f * yy);
    mz[q] = pk2(-2.f * yz, -2.f * yz);
    ny[q] = pk2(n, n);
    ah[q] = pk2(y0.w, y0.w);
  }
  const u64 nq = pk2(-qexp, -qexp);

  RunningSums<P, TPB, KS> run(sk);

  constexpr int Q4 = TJ / 4;  // float4s per row of one record tile
  for (int t = t0; t < t1; t += SUB) {
    __syncthreads();
#pragma unroll
    for (int sub = 0; sub < SUB; ++sub) {
      if (t + sub < t1) {
        const float4* g4 = reinterpret_cast<const float4*>(Xr + (size_t)(t + sub) * 4 * TJ);
        const float4* a4 = reinterpret_cast<const float4*>(XA + (size_t)(t + sub) * 2 * TJ);
#pragma unroll
        for (int u = tid; u < 4 * Q4; u += TPB)                            // rows 0..3
          *reinterpret_cast<float4*>(&sT[u / Q4][sub * TJ + 4 * (u % Q4)]) = g4[u];
#pragma unroll
        for (int u = tid; u < 2 * Q4; u += TPB)                            // rows 4..5
          *reinterpret_cast<float4*>(&sT[4 + u / Q4][sub * TJ + 4 * (u % Q4)]) = a4[u];
      } else {
        for (int u = tid; u < TJ; u += TPB) {
#pragma unroll
          for (int r = 0; r < 5; ++r) sT[r][sub * TJ + u] = 0.f;
          sT[5][sub * TJ + u] = INFINITY;
        }
      }
    }
    __syncthreads();

    u64 aW[P], ax[P], ay[P], az[P];
#pragma unroll
    for (int q = 0; q < P; ++q) aW[q] = ax[q] = ay[q] = az[q] = 0ull;  // +0.0f in both lanes

    // two 4-point steps per unrolled body; one for the 4-point shape with
    // shared-memory sums (its 16 pair updates per step fill 112 registers)
    constexpr int UNR = (KS && P >= 4) ? 1 : 2;
    constexpr int JN = HALF ? TJ / 2 : TJ * SUB;
#pragma unroll UNR
    for (int jq = HALF ? jlo : 0; jq < (HALF ? jlo : 0) + JN; jq += 4) {
      const ulonglong2 X = *reinterpret_cast<const ulonglong2*>(&sT[0][jq]);
      const ulonglong2 Yv = *reinterpret_cast<const ulonglong2*>(&sT[1][jq]);
      const ulonglong2 Z = *reinterpret_cast<const ulonglong2*>(&sT[2][jq]);
      const ulonglong2 N = *reinterpret_cast<const ulonglong2*>(&sT[3][jq]);
      const ulonglong2 Av = *reinterpret_cast<const ulonglong2*>(&sT[4][jq]);
      const ulonglong2 Lv = *reinterpret_cast<const ulonglong2*>(&sT[5][jq]);
#pragma unroll
      for (int q = 0; q < P; ++q)
        pair2<PM>(X.x, Yv.x, Z.x, N.x, Av.x, Lv.x, mx[q], my[q], mz[q], ny[q], ah[q], nq, aW[q], ax[q], ay[q], az[q]);
#pragma unroll
      for (int q = 0; q < P; ++q) {
        if (q < EXO)  // resolved at compile time once the loop is unrolled
          pair2<PM, true>(X.y, Yv.y, Z.y, N.y, Av.y, Lv.y, mx[q], my[q], mz[q], ny[q], ah[q], nq, aW[q], ax[q], ay[q],
                          az[q]);
        else
          pair2<PM>(X.y, Yv.y, Z.y, N.y, Av.y, Lv.y, mx[q], my[q], mz[q], ny[q], ah[q], nq, aW[q], ax[q], ay[q], az[q]);
      }
    }
#pragma unroll
    for (int q = 0; q < P; ++q) run.add(q, aW[q], ax[q], ay[q], az[q]);
  }

  float4* out = outbase + tid;
#pragma unroll
  for (int q = 0; q < P; ++q) out[q * TPB] = run.result(q);
}

// Work item {pair, template block, reference chunk} of a batch: the block's
// template range, tile range, pose and output slot.
template <int P, int TPB>
__device__ __forceinline__ void batch_item(const int4 it, const BatchPair* __restrict__ pairs,
                                           int tiles_per_split, const DevPose* __restrict__ pose,
                                           float4* __restrict__ partial, int& ibase, int& t0, int& t1,
                                           const DevPose*& ps, float4*& outbase) {
  const BatchPair& bp = pairs[it.x];
  const int lt0 = it.z * tiles_per_split;
  const int local = it.y * (TPB * P);
  t0 = (int)bp.xtile0 + lt0;
  t1 = (int)bp.xtile0 + min(bp.ntiles, lt0 + tiles_per_split);
  ibase = (int)bp.ybase + local;
  ps = pose + it.x;
  outbase = partial + bp.pbase + (size_t)it.z * bp.mpad + local;
}

// BATCH = false: one problem, grid (template blocks, reference splits).
// BATCH = true: one block per work item {pair, template block, reference
// chunk} of a batch of independent problems (items[], pairs[], one pose per
// pair); tiles_per_split is then the chunk length in tiles.
// KS, SUB: running sums in shared memory, record tiles staged SUB at a time.
template <int P, int PM, int TPB, int TJ, int MINB, bool BATCH, bool KS = false, int SUB = 1, int EXO = 0,
          bool HALF = false>
__global__ void __launch_bounds__(TPB, MINB)
    force_tile_kernel(const float* __restrict__ Xr, const float* __restrict__ XA, int ntiles,
                      int tiles_per_split, const float4* __restrict__ Y0r, int mpad,
                      const DevPose* __restrict__ pose, float qexp, float4* __restrict__ partial,
                      const int4* __restrict__ items, const BatchPair* __restrict__ pairs) {
  __shared__ __align__(16) float sT[6][TJ * SUB];
  __shared__ float sK[KS ? 8 * P * TPB : 1];
  int ibase, t0, t1;
  const DevPose* ps;
  float4* outbase;
  int jlo = 0;
  if (BATCH) {
    batch_item<P, TPB>(items[blockIdx.x], pairs, tiles_per_split, pose, partial, ibase, t0, t1, ps, outbase);
  } else {
    ibase = blockIdx.x * (TPB * P);
    if (HALF) {  // split y: half y % 2 of tile y / 2
      t0 = blockIdx.y >> 1;
      t1 = t0 + 1;
      jlo = (blockIdx.y & 1) * (TJ / 2);
    } else {
      t0 = blockIdx.y * tiles_per_split;
      t1 = min(ntiles, t0 + tiles_per_split);
    }
    ps = pose;
    outbase = partial + (size_t)blockIdx.y * mpad + ibase;
  }
  force_block<P, PM, TPB, TJ, KS, SUB, EXO, HALF>(sT, sK, Xr, XA, t0, t1, Y0r, ibase, ps, qexp, outbase, jlo);
}

// Persistent form of the batched pass: a grid of resident blocks takes work
// items from a queue in index order (items are sorted longest first, so the
// blocks finish close together: greedy longest-processing-time scheduling).
// *next is the queue head; it must be 0 at launch (the caller clears it).
// Each item's result depends only on the item, so which block takes it does
// not change any bit of the output.  No block waits for another.
template <int P, int PM, int TPB, int TJ, int MINB, bool KS = false, int SUB = 1>
__global__ void __launch_bounds__(TPB, MINB)
    force_batch_persistent_kernel(const float* __restrict__ Xr, const float* __restrict__ XA,
                                  int tiles_per_split, const float4* __restrict__ Y0r,
                                  const DevPose* __restrict__ pose, float qexp, float4* __restrict__ partial,
                                  const int4* __restrict__ items, int nitems, const BatchPair* __restrict__ pairs,
                                  int* __restrict__ next) {
  __shared__ __align__(16) float sT[6][TJ * SUB];
  __shared__ float sK[KS ? 8 * P * TPB : 1];
  __shared__ int s_item;
  for (;;) {
    if (threadIdx.x == 0) s_item = atomicAdd(next, 1);
    __syncthreads();
    const int item = s_item;
    if (item >= nitems) break;
    int ibase, t0, t1;
    const DevPose* ps;
    float4* outbase;
    batch_item<P, TPB>(items[item], pairs, tiles_per_split, pose, partial, ibase, t0, t1, ps, outbase);
    force_block<P, PM, TPB, TJ, KS, SUB>(sT, sK, Xr, XA, t0, t1, Y0r, ibase, ps, qexp, outbase);
    __syncthreads();  // every thread has read s_item before thread 0 takes the next one
  }
}

// Mixed batched pass: each work item takes the shape its pair was planned
// with (BatchPair::shape4) - 4 template points x 128 threads with the running
// sums in shared memory and 512-point stages, the fastest shape per pair
// (the one large templates use), for pairs whose templates fill 512-point
// blocks well, and 2 points x 128 threads for the others, whose templates
// would otherwise be padded to a multiple of 512.  One launch for both
// shapes, so the longest-first item order fills the last wave with the
// shortest items of either kind.  The 2-point shape uses the first half of
// the record stage as its 256-point tile.
template <int PM>
__global__ void __launch_bounds__(128, 3)
    force_batch_mixed_kernel(const float* __restrict__ Xr, const float* __restrict__ XA, int tiles_per_split,
                             const float4* __restrict__ Y0r, const DevPose* __restrict__ pose, float qexp,
                             float4* __restrict__ partial, const int4* __restrict__ items,
                             const BatchPair* __restrict__ pairs) {
  __shared__ __align__(16) float sT[6][FORCE_TJ * 2];
  __shared__ float sK[8 * 4 * 128];
  const int4 it = items[blockIdx.x];
  int ibase, t0, t1;
  const DevPose* ps;
  float4* outbase;
  if (pairs[it.x].shape4) {
    batch_item<4, 128>(it, pairs, tiles_per_split, pose, partial, ibase, t0, t1, ps, outbase);
    force_block<4, PM, 128, FORCE_TJ, true, 2>(sT, sK, Xr, XA, t0, t1, Y0r, ibase, ps, qexp, outbase);
  } else {
    batch_item<2, 128>(it, pairs, tiles_per_split, pose, partial, ibase, t0, t1, ps, outbase);
    float(&s1)[6][FORCE_TJ] = *reinterpret_cast<float(*)[6][FORCE_TJ]>(&sT[0][0]);
    force_block<2, PM, 128, FORCE_TJ, false, 1>(s1, sK, Xr, XA, t0, t1, Y0r, ibase, ps, qexp, outbase);
  }
}

// ---- planning --------------------------------------------------------------

static int force_blocks_per_sm(const ForcePlan& fp);

// Duration, in tiles, of a force grid under greedy dispatch: blocks start in
// split-major order (grid.x fastest), each on the earliest free of `slots`
// resident block slots; blocks of the first splits - 1 splits take d1 tiles,
// those of the last split d2 <= d1.
static double split_makespan(int64_t iblocks, int64_t splits, double d1, double d2, int64_t slots) {
  const int64_t n1 = (splits - 1) * iblocks;
  const int64_t q = n1 / slots, r = n1 % slots;
  double fin = (double)(r > 0 ? q + 1 : q) * d1;
  // after the long blocks: slots - r slots free at q d1, r slots at (q + 1) d1
  const int64_t na = slots - r, nb = r;
  double ta = (double)q * d1, tb = (double)(q + 1) * d1;
  int64_t left = iblocks;
  while (left > 0) {
    if (nb == 0 || ta <= tb) {
      left -= left < na ? left : na;
      fin = fin > ta + d2 ? fin : ta + d2;
      ta += d2;
    } else {
      left -= left < nb ? left : nb;
      fin = fin > tb + d2 ? fin : tb + d2;
      tb += d2;
    }
  }
  return fin;
}

// Work split: template points per thread by size, then the reference split
// length L (tiles per block).  A block stages force_stage_tiles(fp) tiles at
// a time, so L is a multiple of that (an odd L on a two-tile stage computes
// a padded tile: 20% more time at 35k points, where L is 5).  Each candidate
// L is scored by the makespan of its grid under greedy dispatch plus a
// quarter of one block's duration: blocks on different SMs finish at
// different times, so shorter blocks leave a shorter ragged tail (over split
// lengths 2..25 on 20k-50k point problems the score's choice was within 1% of
// the fastest length measured).  The lowest score wins, ties to fewer
// splits.  At most max(16, twelve waves' worth) and 128 splits, and at least
// two tiles per split unless that leaves the grid short of one wave (small
// problems, where a block's sequential walk over its tiles is the launch's
// latency): then down to one tile per split, and to half a tile (fp.half)
// where even that grid fills less than half a wave.
ForcePlan plan_force(int64_t m, int64_t npad, double p, int num_sms, const ForceTuning& tune, int blocks_per_sm) {
  ForcePlan fp;
  fp.pmode = (p == 1.0) ? 1 : (p == 2.0) ? (tune.rsq == 1 ? 4 : 2) : (p == 3.0) ? 3 : 0;
  fp.tile_j = FORCE_TJ;
  // by template size: 4 points per thread in blocks of 128 with the running
  // sums in shared memory (the fastest shape measured for large templates),
  // then 2 and 1 points per thread in blocks of 256
  fp.tpb = 256;
  if (m >= (int64_t)num_sms * 2 * 256 * 4) {
    fp.P = 4;
    fp.tpb = 128;
  } else if (m >= (int64_t)num_sms * 256 * 2) {
    fp.P = 2;
  } else {
    fp.P = 1;
  }
  if (m < 4096) fp.tpb = 128;
  if (tune.P == 1 || tune.P == 2 || tune.P == 4) fp.P = tune.P;
  if (tune.tpb == 128 || tune.tpb == 256) fp.tpb = tune.tpb;
  const int occ = tune.occ >= 0 ? tune.occ : (fp.P == 4 && fp.tpb == 128) ? 2 : 0;
  if (occ == 1)
    fp.occ = (fp.tpb == 256 && fp.P == 4) ? 0 : 1;
  else if (occ == 2)
    fp.occ = ((fp.P == 4 && fp.tpb == 128) || (fp.P == 2 && fp.tpb == 256)) ? 2 : 0;
  else
    fp.occ = 0;
  fp.ex2poly = (fp.pmode == 2 && fp.occ == 2) ? (tune.ex2poly < fp.P ? tune.ex2poly : fp.P) : 0;
  const int64_t per_block = (int64_t)fp.tpb * fp.P;
  fp.iblocks = (int)((m + per_block - 1) / per_block);
  const int64_t ntiles = npad / FORCE_TJ > 0 ? npad / FORCE_TJ : 1;
  const int64_t slots = (int64_t)num_sms * (blocks_per_sm > 0 ? blocks_per_sm : force_blocks_per_sm(fp));
  const int64_t sub = force_stage_tiles(fp);
  auto up = [](int64_t a, int64_t b) { return (a + b - 1) / b; };
  int64_t L = 0;
  if (tune.splits > 0) {
    // an explicit split count is taken as given (lengths not rounded)
    L = up(ntiles, tune.splits < ntiles ? tune.splits : ntiles);
  } else {
    int64_t S_max = up(12 * slots, fp.iblocks);
    if (S_max < 16) S_max = 16;
    if (S_max > 128) S_max = 128;
    const int64_t floor_len = (int64_t)fp.iblocks * up(ntiles, 2) < slots ? sub : (sub > 2 ? sub : 2);
    int64_t L_min = up(ntiles, S_max) > floor_len ? up(ntiles, S_max) : floor_len;
    L_min = up(L_min, sub) * sub;
    double best = 0.0;
    int64_t last = -1;
    for (int64_t S = 1; S <= S_max; ++S) {
      const int64_t len = up(up(ntiles, S), sub) * sub;
      if (len < L_min || len == last) continue;
      last = len;
      const int64_t splits = up(ntiles, len);
      const int64_t tail = up(ntiles - (splits - 1) * len, sub) * sub;
      const double score = split_makespan(fp.iblocks, splits, (double)len, (double)tail, slots) + 0.25 * (double)len;
      if (L == 0 || score < best - 1e-9) {
        best = score;
        L = len;
      }
    }
    if (L == 0) L = L_min;
  }
  fp.tiles_per_split = (int)L;
  fp.splits = (int)up(ntiles, L);
  // the smallest problems (1 point x 128 threads, one tile per split, the
  // grid under half a wave): split every tile in two, halving the dependent
  // steps of each thread
  fp.half = 0;
  if (tune.splits == 0 && L == 1 && fp.P == 1 && fp.tpb == 128 && fp.occ == 0 &&
      2 * (int64_t)fp.iblocks * ntiles <= slots) {
    fp.half = 1;
    fp.splits = (int)(2 * ntiles);
  }
  return fp;
}

int64_t force_mpad(int64_t m, const ForcePlan& fp) {
  const int64_t per_block = (int64_t)fp.tpb * fp.P;
  int64_t mp = (m + per_block - 1) / per_block * per_block;
  // the combine kernel works in blocks of 256
  return (mp + 255) / 256 * 256;
}

template <int P, int PM, int TPB, int MINB, bool KS, int SUB, int EXO, bool HALF = false>
static void launch_force_t(cudaStream_t st, const ForcePlan& fp, const float4* Xr,
                           const float2* XA, int ntiles, const float4* Y0r, int mpad,
                           const DevPose* pose, float qexp, float4* partial) {
  dim3 grid(fp.iblocks, fp.splits);
  force_tile_kernel<P, PM, TPB, FORCE_TJ, MINB, false, KS, SUB, EXO, HALF><<<grid, TPB, 0, st>>>(
      reinterpret_cast<const float*>(Xr), reinterpret_cast<const float*>(XA), ntiles,
      fp.tiles_per_split, Y0r, mpad, pose, qexp, partial, nullptr, nullptr);
}

// Dispatch on (points per thread, threads, occupancy variant): calls
// f.template operator()<P, TPB, MINB, KS, SUB>() for the kernel instance of
// the plan.  Variant 2 keeps the running sums in shared memory and stages
// two record tiles (512 reference points) at a time.
template <class F>
static int with_shape(const ForcePlan& fp, const F& f) {
  const bool hi = fp.occ == 1;
  if (fp.occ == 2) {
    if (fp.P == 4 && fp.tpb == 128) {
      if (fp.ex2poly == 1) return f.template operator()<4, 128, 3, true, 2, 1>();
      if (fp.ex2poly == 2) return f.template operator()<4, 128, 3, true, 2, 2>();
      return f.template operator()<4, 128, 3, true, 2>();
    }
    if (fp.P == 2 && fp.tpb == 256) {
      if (fp.ex2poly == 1) return f.template operator()<2, 256, 2, true, 2, 1>();
      if (fp.ex2poly == 2) return f.template operator()<2, 256, 2, true, 2, 2>();
      return f.template operator()<2, 256, 2, true, 2>();
    }
  }
  if (fp.tpb == 256) {
    if (fp.P == 4) return f.template operator()<4, 256, 2, false, 1>();
    if (fp.P == 2) return hi ? f.template operator()<2, 256, 3, false, 1>() : f.template operator()<2, 256, 2, false, 1>();
    return hi ? f.template operator()<1, 256, 4, false, 1>() : f.template operator()<1, 256, 2, false, 1>();
  }
  if (fp.P == 4) return hi ? f.template operator()<4, 128, 4, false, 1>() : f.template operator()<4, 128, 2, false, 1>();
  if (fp.P == 2) return hi ? f.template operator()<2, 128, 4, false, 1>() : f.template operator()<2, 128, 2, false, 1>();
  return hi ? f.template operator()<1, 128, 4, false, 1>() : f.template operator()<1, 128, 2, false, 1>();
}

template <int PM>
struct LaunchShape {
  cudaStream_t st;
  const ForcePlan& fp;
  const float4* Xr;
  const float2* XA;
  int ntiles;
  const float4* Y0r;
  int mpad;
  const DevPose* pose;
  float qexp;
  float4* partial;
  template <int P, int TPB, int MINB, bool KS, int SUB, int EXO = 0>
  int operator()() const {
    // the FP32-pipe exponential exists for p = 2 (sqrt form) only
    constexpr int E = PM == 2 ? EXO : 0;
    if constexpr (P == 1 && TPB == 128 && MINB == 2 && !KS && SUB == 1) {
      if (fp.half) {
        launch_force_t<P, PM, TPB, MINB, KS, SUB, E, true>(st, fp, Xr, XA, ntiles, Y0r, mpad, pose, qexp, partial);
        return 0;
      }
    }
    launch_force_t<P, PM, TPB, MINB, KS, SUB, E>(st, fp, Xr, XA, ntiles, Y0r, mpad, pose, qexp, partial);
    return 0;
  }
};

template <int PM>
static void launch_force_pm(cudaStream_t st, const ForcePlan& fp, const float4* Xr,
                            const float2* XA, int ntiles, const float4* Y0r, int mpad,
                            const DevPose* pose, float qexp, float4* partial) {
  with_shape(fp, LaunchShape<PM>{st, fp, Xr, XA, ntiles, Y0r, mpad, pose, qexp, partial});
}

template <int PM>
struct OccShape {
  template <int P, int TPB, int MINB, bool KS, int SUB, int EXO = 0>
  int operator()() const {
    constexpr int E = PM == 2 ? EXO : 0;
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(
            &nb, force_tile_kernel<P, PM, TPB, FORCE_TJ, MINB, false, KS, SUB, E>, TPB, 0) != cudaSuccess) {
      cudaGetLastError();
      return 2;
    }
    return nb > 0 ? nb : 1;
  }
};

template <int PM>
static int blocks_per_sm_pm(const ForcePlan& fp) {
  return with_shape(fp, OccShape<PM>{});
}

static int force_blocks_per_sm(const ForcePlan& fp) {
  switch (fp.pmode) {
    case 1: return blocks_per_sm_pm<1>(fp);
    case 2: return blocks_per_sm_pm<2>(fp);
    case 3: return blocks_per_sm_pm<3>(fp);
    case 4: return blocks_per_sm_pm<4>(fp);
    default: return blocks_per_sm_pm<0>(fp);
  }
}

cudaError_t launch_force(Launch L, const ForcePlan& fp, const float4* Xr, const float2* XA,
                         int ntiles, const float4* Y0r, int mpad, const DevPose* pose, float qexp,
                         float4* partial) {
  switch (fp.pmode) {
    case 1: launch_force_pm<1>(L.stream, fp, Xr, XA, ntiles, Y0r, mpad, pose, qexp, partial); break;
    case 2: launch_force_pm<2>(L.stream, fp, Xr, XA, ntiles, Y0r, mpad, pose, qexp, partial); break;
    case 3: launch_force_pm<3>(L.stream, fp, Xr, XA, ntiles, Y0r, mpad, pose, qexp, partial); break;
    case 4: launch_force_pm<4>(L.stream, fp, Xr, XA, ntiles, Y0r, mpad, pose, qexp, partial); break;
    default: launch_force_pm<0>(L.stream, fp, Xr, XA, ntiles, Y0r, mpad, pose, qexp, partial); break;
  }
  if (L.counter) ++*L.counter;
  return cudaGetLastError();
}

// Batched force pass, P template points per thread: one block per item
// (grid == 0), or a persistent grid of `grid` resident blocks taking items
// from the queue head *next, which is cleared first.  P = 1, 2: 128 threads.
// P = 4: 64 threads (a 256-point template block, as for P = 2), the
// shared-memory running sums and 512-point stages, 6 blocks per SM.
template <int P>
struct BatchShape {
  static constexpr bool KS = P == 4;
  static constexpr int SUB = P == 4 ? 2 : 1;
  static constexpr int TPB = P == 4 ? 64 : 128;
  static constexpr int MINB = P == 4 ? 6 : 2;
};

int batch_block_threads(int P) { return P == 4 ? BatchShape<4>::TPB : BatchShape<1>::TPB; }

// Shape of pair template of m points in the mixed batched pass: the 4-point
// shape (512-point blocks) unless its padding costs more than its speed
// (measured per pair on GB300: 9.0 against 8.5 pairs per clock per SM for
// the 2-point shape with 256-point blocks).
bool batch_pair_shape4(int64_t m) {
  const int64_t pad4 = (m + 511) / 512 * 512;
  const int64_t pad2 = (m + 255) / 256 * 256;
  return (double)pad4 * 8.5 <= (double)pad2 * 9.0;
}

template <int P, int PM>
static void launch_force_batch_p(cudaStream_t st, int nitems, const int4* items, const BatchPair* pairs,
                                 const float4* Xr, const float2* XA, const float4* Y0r, const DevPose* poses,
                                 float qexp, float4* partial, int chunk_tiles, int grid, int* next) {
  const float* xr = reinterpret_cast<const float*>(Xr);
  const float* xa = reinterpret_cast<const float*>(XA);
  if constexpr (P == 0) {
    force_batch_mixed_kernel<PM><<<nitems, 128, 0, st>>>(xr, xa, chunk_tiles, Y0r, poses, qexp, partial, items,
                                                         pairs);
  } else {
    using B = BatchShape<P>;
    if (grid <= 0)
      force_tile_kernel<P, PM, B::TPB, FORCE_TJ, B::MINB, true, B::KS, B::SUB><<<nitems, B::TPB, 0, st>>>(
          xr, xa, 0, chunk_tiles, Y0r, 0, poses, qexp, partial, items, pairs);
    else
      force_batch_persistent_kernel<P, PM, B::TPB, FORCE_TJ, B::MINB, B::KS, B::SUB>
          <<<grid < nitems ? grid : nitems, B::TPB, 0, st>>>(xr, xa, chunk_tiles, Y0r, poses, qexp, partial, items,
                                                            nitems, pairs, next);
  }
}

template <int PM>
static void launch_force_batch_pm(cudaStream_t st, int P, int nitems, const int4* items, const BatchPair* pairs,
                                  const float4* Xr, const float2* XA, const float4* Y0r, const DevPose* poses,
                                  float qexp, float4* partial, int chunk_tiles, int grid, int* next) {
  if (P == 0)
    launch_force_batch_p<0, PM>(st, nitems, items, pairs, Xr, XA, Y0r, poses, qexp, partial, chunk_tiles, 0, next);
  else if (P == 4)
    launch_force_batch_p<4, PM>(st, nitems, items, pairs, Xr, XA, Y0r, poses, qexp, partial, chunk_tiles, grid, next);
  else if (P == 2)
    launch_force_batch_p<2, PM>(st, nitems, items, pairs, Xr, XA, Y0r, poses, qexp, partial, chunk_tiles, grid, next);
  else
    launch_force_batch_p<1, PM>(st, nitems, items, pairs, Xr, XA, Y0r, poses, qexp, partial, chunk_tiles, grid, next);
}

cudaError_t launch_force_batch(Launch L, int pmode, int P, int nitems, const int4* items, const BatchPair* pairs,
                               const float4* Xr, const float2* XA, const float4* Y0r, const DevPose* poses,
                               float qexp, float4* partial, int chunk_tiles, int grid, int* next) {
  if (nitems <= 0) return cudaSuccess;
  if (grid > 0) {
    if (!next) return cudaErrorInvalidValue;
    const cudaError_t e = cudaMemsetAsync(next, 0, sizeof(int), L.stream);
    if (e != cudaSuccess) return e;
  }
  switch (pmode) {
    case 1: launch_force_batch_pm<1>(L.stream, P, nitems, items, pairs, Xr, XA, Y0r, poses, qexp, partial, chunk_tiles, grid, next); break;
    case 2: launch_force_batch_pm<2>(L.stream, P, nitems, items, pairs, Xr, XA, Y0r, poses, qexp, partial, chunk_tiles, grid, next); break;
    case 3: launch_force_batch_pm<3>(L.stream, P, nitems, items, pairs, Xr, XA, Y0r, poses, qexp, partial, chunk_tiles, grid, next); break;
    case 4: launch_force_batch_pm<4>(L.stream, P, nitems, items, pairs, Xr, XA, Y0r, poses, qexp, partial, chunk_tiles, grid, next); break;
    default: launch_force_batch_pm<0>(L.stream, P, nitems, items, pairs, Xr, XA, Y0r, poses, qexp, partial, chunk_tiles, grid, next); break;
  }
  if (L.counter) ++*L.counter;
  return cudaGetLastError();
}

// Resident blocks of the persistent batched force kernel on the current device.
template <int PM>
static cudaError_t batch_slots_pm(int P, int* slots) {
  int dev = 0, sms = 0, nb = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess) {
    if (P == 4)
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
          &nb, force_batch_persistent_kernel<4, PM, BatchShape<4>::TPB, FORCE_TJ, BatchShape<4>::MINB, true, 2>,
          BatchShape<4>::TPB, 0);
    else if (P == 2)
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, force_batch_persistent_kernel<2, PM, 128, FORCE_TJ, 2>, 128, 0);
    else
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, force_batch_persistent_kernel<1, PM, 128, FORCE_TJ, 2>, 128, 0);
  }
  if (e != cudaSuccess) return e;
  *slots = sms * (nb > 0 ? nb : 1);
  return cudaSuccess;
}

cudaError_t force_batch_slots(int pmode, int P, int* slots) {
  switch (pmode) {
    case 1: return batch_slots_pm<1>(P, slots);
    case 2: return batch_slots_pm<2>(P, slots);
    case 3: return batch_slots_pm<3>(P, slots);
    case 4: return batch_slots_pm<4>(P, slots);
    default: return batch_slots_pm<0>(P, slots);
  }
}

// ---- p = 3: moments of the pair weights over the reference ------------------
// For p = 3, w_ij = g_ij d_ij^2 with g_ij = aX_j s_ij (or s_ij) independent of
// the pose, and d^2 = |Y|^2 - 2 Y.X + |X|^2, so the per-point sums expand into
// moments over j of g alone (X' in the frame centred on the reference mean):
//   sum w   = |Y|^2 M0 - 2 Y.M1 + m2,
//   sum w X = |Y|^2 M1 - 2 M2 Y + m3,
// with M0 = sum g, M1 = sum g X', M2 = sum g X' X'^T, m2 = sum g |X'|^2,
// m3 = sum g |X'|^2 X'.  One pass computes them (packed float32 per tile,
// Kahan-compensated float32 across tiles), after which an iteration is O(M).
constexpr int MOM_TPB = 256;
constexpr int NMOM = 14;  // M0, M1[3], M2[6] (xx xy xz yy yz zz), m2, m3[3]

// One packed moment update: reference points (j, j+1) against one template
// point (ah = its a_hat in both lanes): g = 2^-(u^2 - L) (the pair factor of
// the force kernel), then g, g X', g X' X'^T, g |X'|^2, g |X'|^2 X' added to
// the 14 packed accumulators m[].
__device__ __forceinline__ void moment2(u64 xv, u64 yv, u64 zv, u64 nv, u64 av, u64 lv, u64 ah, u64 (&m)[NMOM]) {
  const u64 u = sub2(av, ah);
  float e0, e1;
  upk2(fma2(u, u, lv), e0, e1);
  const u64 g = pk2(ex2_neg(e0), ex2_neg(e1));
  const u64 gx = mul2(g, xv), gy = mul2(g, yv), gz = mul2(g, zv), gn = mul2(g, nv);
  m[0] = add2(m[0], g);
  m[1] = add2(m[1], gx);
  m[2] = add2(m[2], gy);
  m[3] = add2(m[3], gz);
  m[4] = fma2(gx, xv, m[4]);
  m[5] = fma2(gx, yv, m[5]);
  m[6] = fma2(gx, zv, m[6]);
  m[7] = fma2(gy, yv, m[7]);
  m[8] = fma2(gy, zv, m[8]);
  m[9] = fma2(gz, zv, m[9]);
  m[10] = add2(m[10], gn);
  m[11] = fma2(gn, xv, m[11]);
  m[12] = fma2(gn, yv, m[12]);
  m[13] = fma2(gn, zv, m[13]);
}

// Per template point, the 14 moments over reference tiles [t0, t1) of one
// split: each tile's sums in packed float32 (two reference points per
// instruction, 128-bit shared-memory broadcasts of four points), added to
// float32 running sums with Kahan compensation; the split's result is
// written as doubles.  Padding records have -L = +inf, so g = 0.
__global__ void __launch_bounds__(MOM_TPB)
    moments_kernel(const float* __restrict__ Xr, const float* __restrict__ XA, int ntiles, int tiles_per_split,
                   const float4* __restrict__ Y0r, int mpad, double* __restrict__ mpart) {
  __shared__ __align__(16) float sT[6][FORCE_TJ];
  const int i = blockIdx.x * MOM_TPB + threadIdx.x;
  const int split = blockIdx.y;
  const float a = Y0r[i].w;
  const u64 ah = pk2(a, a);
  float hs[NMOM], cs[NMOM];
#pragma unroll
  for (int q = 0; q < NMOM; ++q) hs[q] = cs[q] = 0.f;
  const int t0 = split * tiles_per_split;
  const int t1 = min(ntiles, t0 + tiles_per_split);
  constexpr int Q4 = FORCE_TJ / 4;
  for (int t = t0; t < t1; ++t) {
    __syncthreads();
    const float4* g4 = reinterpret_cast<const float4*>(Xr + (size_t)t * 4 * FORCE_TJ);
    const float4* a4 = reinterpret_cast<const float4*>(XA + (size_t)t * 2 * FORCE_TJ);
    for (int u = threadIdx.x; u < 4 * Q4; u += MOM_TPB) *reinterpret_cast<float4*>(&sT[u / Q4][4 * (u % Q4)]) = g4[u];
    for (int u = threadIdx.x; u < 2 * Q4; u += MOM_TPB)
      *reinterpret_cast<float4*>(&sT[4 + u / Q4][4 * (u % Q4)]) = a4[u];
    __syncthreads();
    u64 m[NMOM];
#pragma unroll
    for (int q = 0; q < NMOM; ++q) m[q] = 0ull;
#pragma unroll 2
    for (int jq = 0; jq < FORCE_TJ; jq += 4) {
      const ulonglong2 X = *reinterpret_cast<const ulonglong2*>(&sT[0][jq]);
      const ulonglong2 Yv = *reinterpret_cast<const ulonglong2*>(&sT[1][jq]);
      const ulonglong2 Z = *reinterpret_cast<const ulonglong2*>(&sT[2][jq]);
      const ulonglong2 N = *reinterpret_cast<const ulonglong2*>(&sT[3][jq]);
      const ulonglong2 Av = *reinterpret_cast<const ulonglong2*>(&sT[4][jq]);
      const ulonglong2 Lv = *reinterpret_cast<const ulonglong2*>(&sT[5][jq]);
      moment2(X.x, Yv.x, Z.x, N.x, Av.x, Lv.x, ah, m);
      moment2(X.y, Yv.y, Z.y, N.y, Av.y, Lv.y, ah, m);
    }
#pragma unroll
    for (int q = 0; q < NMOM; ++q) {
      float l0, l1;
      upk2(m[q], l0, l1);
      kahan_add(hs[q], cs[q], l0 + l1);
    }
  }
  double* out = mpart + ((size_t)split * mpad + i) * NMOM;
#pragma unroll
  for (int q = 0; q < NMOM; ++q) out[q] = (double)hs[q] - (double)cs[q];
}

// Per-point moments: the splits added in order.
__global__ void moments_reduce_kernel(const double* __restrict__ mpart, int S, int mpad, int m,
                                      double* __restrict__ mom) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m) return;
  double acc[NMOM];
  for (int q = 0; q < NMOM; ++q) acc[q] = 0.0;
  for (int s = 0; s < S; ++s)
    for (int q = 0; q < NMOM; ++q) acc[q] += mpart[((size_t)s * mpad + i) * NMOM + q];
  for (int q = 0; q < NMOM; ++q) mom[(size_t)i * NMOM + q] = acc[q];
}

// The combine of an iteration from the moments (same per-block output as
// combine_kernel).
__global__ void __launch_bounds__(RED_THREADS)
    combine_moments_kernel(const double* __restrict__ mom, int m, const float4* __restrict__ Y0r,
                           const double* __restrict__ aY64, int g_mode, const DevPose* __restrict__ ps,
                           float4* __restrict__ f4out, double* __restrict__ blockpart) {
  __shared__ double sh[13][RED_THREADS];
  const int i = blockIdx.x * RED_THREADS + threadIdx.x;
  double v[13];
#pragma unroll
  for (int q = 0; q < 13; ++q) v[q] = 0.0;
  if (i < m) {
    const double* M = mom + (size_t)i * NMOM;
    float A[9], b[3];
#pragma unroll
    for (int q = 0; q < 9; ++q) A[q] = ps->A[q];
#pragma unroll
    for (int q = 0; q < 3; ++q) b[q] = ps->b[q];
    float yx, yy, yz;
    template_point(Y0r[i], A, b, yx, yy, yz);
    const double Y[3] = {yx, yy, yz};
    const double ny = Y[0] * Y[0] + Y[1] * Y[1] + Y[2] * Y[2];
    const double W = ny * M[0] - 2.0 * (Y[0] * M[1] + Y[1] * M[2] + Y[2] * M[3]) + M[10];
    const double M2Y[3] = {M[4] * Y[0] + M[5] * Y[1] + M[6] * Y[2], M[5] * Y[0] + M[7] * Y[1] + M[8] * Y[2],
                           M[6] * Y[0] + M[8] * Y[1] + M[9] * Y[2]};
    const double S[3] = {ny * M[1] - 2.0 * M2Y[0] + M[11], ny * M[2] - 2.0 * M2Y[1] + M[12],
                         ny * M[3] - 2.0 * M2Y[2] + M[13]};
    const double ay = g_mode == 1 ? aY64[i] : 1.0;
    const double f[3] = {ay * (S[0] - Y[0] * W), ay * (S[1] - Y[1] * W), ay * (S[2] - Y[2] * W)};
    const double Wi = ay * W;
    const double c[3] = {Y[0] - ps->ybs[0], Y[1] - ps->ybs[1], Y[2] - ps->ybs[2]};
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

int moments_splits(int ntiles, int num_sms, int64_t mpad) {
  const int64_t blocks = (mpad + MOM_TPB - 1) / MOM_TPB;
  int64_t S = (num_sms * 4 * 4 + blocks - 1) / blocks;
  if (S > ntiles) S = ntiles;
  if (S < 1) S = 1;
  if (S > 32) S = 32;
  return (int)S;
}

cudaError_t launch_moments(Launch L, const float4* Xr, const float2* XA, int ntiles, const float4* Y0r, int mpad,
                           int m, int S, double* mpart, double* mom) {
  const int tps = (ntiles + S - 1) / S;
  const int splits = (ntiles + tps - 1) / tps;
  moments_kernel<<<dim3((mpad + MOM_TPB - 1) / MOM_TPB, splits), MOM_TPB, 0, L.stream>>>(
      reinterpret_cast<const float*>(Xr), reinterpret_cast<const float*>(XA), ntiles, tps, Y0r, mpad, mpart);
  moments_reduce_kernel<<<(m + 255) / 256, 256, 0, L.stream>>>(mpart, splits, mpad, m, mom);
  if (L.counter) *L.counter += 2;
  return cudaGetLastError();
}

cudaError_t launch_combine_moments(Launch L, const double* mom, int m, int mpad, const float4* Y0r,
                                   const double* aY64, int g_mode, const DevPose* pose, float4* f4out,
                                   double* blockpart) {
  combine_moments_kernel<<<combine_blocks(mpad), RED_THREADS, 0, L.stream>>>(mom, m, Y0r, aY64, g_mode, pose, f4out,
                                                                              blockpart);
  if (L.counter) ++*L.counter;
  return cudaGetLastError();
}

// ---- combine: splits -> per-point force -> per-block (F, W, T) -------------
// A block covers 256 template slots, PPT points per thread.  Per
// point, the split partials are added with Kahan compensation and
// f = aY (S - Y' W) is formed with an exact product (fma) and an exact sum,
// so f is as accurate as float allows even when S and Y' W nearly cancel;
// f (x) c and the other block terms are FP32 products of accurate factors.  A
// thread's points are added in FP32, and every sum across threads and
// blocks is FP64 in a fixed order.  (FP64 arithmetic per point would make
// this kernel FP64-bound: GB300 issues FP64 at a small fraction of FP32.)
// PPT = 4 points per thread (64 threads) where the grid is large; PPT = 1
// (256 threads) for small templates, where a thread's points are sequential
// trips to memory and few threads run per SM.
constexpr int CMB_SLOTS = 256;           // template slots per block
constexpr int CMB_SMALL_BLOCKS = 1024;   // grids of fewer blocks take PPT = 1

// BATCH = true: block b belongs to pair cpair[b]; its 256 template slots are
// that pair's slots (b - cblk0) * 256 + threadIdx.x + (256 / PPT) k, k < PPT.
template <bool BATCH, int PPT>
__global__ void __launch_bounds__(CMB_SLOTS / PPT, 2 * PPT)
    combine_kernel(const float4* __restrict__ partial, int S, int mpad, int m,
                   const float4* __restrict__ Y0r, const float* __restrict__ aY32, int g_mode,
                   const DevPose* __restrict__ pose, float4* __restrict__ f4out,
                   double* __restrict__ blockpart, const int* __restrict__ cpair,
                   const BatchPair* __restrict__ pairs) {
  constexpr int TPB = CMB_SLOTS / PPT;
  __shared__ double sh[TPB / 32][16];
  int i0, mm, SS;
  size_t pstride;
  const float4* pbase;
  const float4* ybase;
  const float* abase;
  const DevPose* ps;
  if (BATCH) {
    const int p = cpair[blockIdx.x];
    const BatchPair& bp = pairs[p];
    i0 = (blockIdx.x - bp.cblk0) * CMB_SLOTS;
    mm = (int)bp.m;
    SS = bp.chunks;
    pstride = (size_t)bp.mpad;
    pbase = partial + bp.pbase;
    ybase = Y0r + bp.ybase;
    abase = aY32 + bp.y0;
    ps = pose + p;
  } else {
    i0 = blockIdx.x * CMB_SLOTS;
    mm = m;
    SS = S;
    pstride = (size_t)mpad;
    pbase = partial;
    ybase = Y0r;
    abase = aY32;
    ps = pose;
  }
  const PointFrame fr(ps);
  float acc[13];
#pragma unroll
  for (int q = 0; q < 13; ++q) acc[q] = 0.f;
#pragma unroll
  for (int k = 0; k < PPT; ++k) {
    const int i = i0 + k * TPB + threadIdx.x;
    if (i < mm) point_force(pbase, pstride, SS, i, ybase[i], g_mode == 1 ? abase[i] : 1.f, fr, acc, f4out);
  }
  double v[16];
#pragma unroll
  for (int q = 0; q < 13; ++q) v[q] = (double)acc[q];
  v[13] = v[14] = v[15] = 0.0;
  warp_reduce16(v);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if ((lane & 1) == 0) sh[warp][warp_reduce16_slot(lane)] = v[0];
  __syncthreads();
  if (threadIdx.x < 13) {
    double t = sh[0][threadIdx.x];
#pragma unroll
    for (int w = 1; w < TPB / 32; ++w) t += sh[w][threadIdx.x];
    blockpart[(size_t)blockIdx.x * 13 + threadIdx.x] = t;
  }
}

int combine_blocks(int64_t mpad) { return (int)((mpad + CMB_SLOTS - 1) / CMB_SLOTS); }

cudaError_t launch_combine(Launch L, const float4* partial, int S, int mpad, int m,
                           const float4* Y0r, const float* aY32, int g_mode, const DevPose* pose,
                           float4* f4out, double* blockpart) {
  const int nb = combine_blocks(mpad);
  if (nb < CMB_SMALL_BLOCKS)
    combine_kernel<false, 1><<<nb, CMB_SLOTS, 0, L.stream>>>(partial, S, mpad, m, Y0r, aY32, g_mode, pose, f4out,
                                                             blockpart, nullptr, nullptr);
  else
    combine_kernel<false, 4><<<nb, CMB_SLOTS / 4, 0, L.stream>>>(partial, S, mpad, m, Y0r, aY32, g_mode, pose,
                                                                 f4out, blockpart, nullptr, nullptr);
  if (L.counter) ++*L.counter;
  return cudaGetLastError();
}

cudaError_t launch_combine_batch(Launch L, int nblocks, const int* cpair, const BatchPair* pairs,
                                 const float4* partial, const float4* Y0r, const float* aY32, int g_mode,
                                 const DevPose* poses, double* blockpart) {
  if (nblocks <= 0) return cudaSuccess;
  combine_kernel<true, 4><<<nblocks, CMB_SLOTS / 4, 0, L.stream>>>(partial, 0, 0, 0, Y0r, aY32, g_mode, poses,
                                                                   nullptr, blockpart, cpair, pairs);
  if (L.counter) ++*L.counter;
  return cudaGetLastError();
}

}  // namespace scgr
