// Throughput microbenchmarks of the units the force kernel is bound by: the
// FP32 FMA pipe (scalar FFMA and packed fma.f32x2) and the special-function
// unit (ex2, sqrt, lg2, rsqrt, and ex2 mixed with rsqrt).  Each thread runs 8 independent dependency chains so
// that latency is hidden; the grid fills every SM.  The results give the
// measured denominators of the force kernel's roofline.
#include <cuda_runtime.h>

#include <cstdint>

#include "common.cuh"
#include "scgr.h"

namespace {

constexpr int MB_CHAINS = 8;
constexpr int MB_ITERS = 4096;
constexpr int MB_TPB = 256;

__device__ __forceinline__ unsigned long long mb_fma2(unsigned long long a, unsigned long long b,
                                                      unsigned long long c) {
  unsigned long long d;
  asm volatile("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}

template <int KIND>
__global__ void __launch_bounds__(MB_TPB) microbench_kernel(float* __restrict__ out, float a, float b) {
  float x[MB_CHAINS];
  unsigned long long y[MB_CHAINS];
#pragma unroll
  for (int c = 0; c < MB_CHAINS; ++c) {
    x[c] = a + 0.001f * c + 1e-7f * threadIdx.x;
    y[c] = ((unsigned long long)__float_as_uint(x[c]) << 32) | __float_as_uint(x[c] + 0.5f);
  }
  const unsigned long long a2 = ((unsigned long long)__float_as_uint(a) << 32) | __float_as_uint(a);
  const unsigned long long b2 = ((unsigned long long)__float_as_uint(b) << 32) | __float_as_uint(b);
  for (int it = 0; it < MB_ITERS; ++it) {
#pragma unroll
    for (int c = 0; c < MB_CHAINS; ++c) {
      if (KIND == 0) {
        x[c] = fmaf(x[c], a, b);
      } else if (KIND == 1) {
        y[c] = mb_fma2(y[c], a2, b2);
      } else if (KIND == 2) {
        float r;
        asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(-x[c]));
        x[c] = r;
      } else if (KIND == 3) {
        float r;
        asm volatile("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x[c]));
        x[c] = r;
      } else if (KIND == 4) {
        float r;
        asm volatile("lg2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x[c]));
        x[c] = r;
      } else if (KIND == 5) {
        float r;
        asm volatile("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x[c]));
        x[c] = r;
      } else if (KIND == 7) {
        // the force kernel's instruction mix: 6 packed FMAs, one ex2 and one
        // sqrt per step.  If the FP32 pipe and the special-function unit
        // overlapped perfectly this would run at the special-function bound
        // (12 unit cycles per 32 steps); if a packed FMA holds the issue
        // port for two cycles, at 14 cycles.
#pragma unroll
        for (int f = 0; f < 6; ++f) y[c] = mb_fma2(y[c], a2, b2);
        float r, w;
        asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(-x[c]));
        asm volatile("sqrt.approx.ftz.f32 %0, %1;" : "=f"(w) : "f"(r));
        x[c] = w;
      } else {
        // ex2 on even chains, rsqrt on odd ones: whether the two share one unit
        float r;
        if (c % 2 == 0)
          asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(-x[c]));
        else
          asm volatile("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x[c]));
        x[c] = r;
      }
    }
  }
  float s = 0.f;
#pragma unroll
  for (int c = 0; c < MB_CHAINS; ++c) s += x[c] + __uint_as_float((unsigned)(y[c] & 0xffffffffu));
  out[blockIdx.x * MB_TPB + threadIdx.x] = s;
}

}  // namespace

// kind: 0 FFMA, 1 packed fma.f32x2, 2 MUFU ex2, 3 MUFU sqrt, 4 MUFU lg2, 5 MUFU rsqrt,
// 6 ex2 and rsqrt interleaved, 7 the force kernel's mix (6 fma.f32x2 + ex2 + sqrt;
// lane_ops counts steps).
// lane_ops: FP32 lane operations (an f32x2 FMA counts 2) or MUFU results;
// ms: device time of one launch on `out_dev` (blocks x 256 floats of scratch
// supplied by the caller, blocks = 8 x SM count).
extern "C" scgr_status scgr_microbench(int kind, int blocks, float* out_dev, void* cuda_stream,
                                       int64_t* lane_ops, double* ms) {
  if (!out_dev || !lane_ops || !ms || blocks < 1 || kind < 0 || kind > 7) return SCGR_ERR_INVALID_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return SCGR_ERR_CUDA;
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return SCGR_ERR_CUDA;
  }
  float best = 1e30f;
  for (int rep = 0; rep < 3; ++rep) {
    cudaEventRecord(e0, st);
    switch (kind) {
      case 0: microbench_kernel<0><<<blocks, MB_TPB, 0, st>>>(out_dev, 0.999f, 1e-3f); break;
      case 1: microbench_kernel<1><<<blocks, MB_TPB, 0, st>>>(out_dev, 0.999f, 1e-3f); break;
      case 2: microbench_kernel<2><<<blocks, MB_TPB, 0, st>>>(out_dev, 0.5f, 0.f); break;
      case 3: microbench_kernel<3><<<blocks, MB_TPB, 0, st>>>(out_dev, 1.5f, 0.f); break;
      case 4: microbench_kernel<4><<<blocks, MB_TPB, 0, st>>>(out_dev, 1.5f, 0.f); break;
      case 5: microbench_kernel<5><<<blocks, MB_TPB, 0, st>>>(out_dev, 1.5f, 0.f); break;
      case 6: microbench_kernel<6><<<blocks, MB_TPB, 0, st>>>(out_dev, 1.5f, 0.f); break;
      default: microbench_kernel<7><<<blocks, MB_TPB, 0, st>>>(out_dev, 0.5f, 1e-3f); break;
    }
    cudaEventRecord(e1, st);
    if (cudaEventSynchronize(e1) != cudaSuccess) {
      cudaGetLastError();
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
      return SCGR_ERR_CUDA;
    }
    float t = 0.f;
    cudaEventElapsedTime(&t, e0, e1);
    if (t < best) best = t;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  const int64_t per_thread = (int64_t)MB_ITERS * MB_CHAINS * (kind == 1 ? 2 : 1);
  *lane_ops = per_thread * blocks * MB_TPB;
  *ms = best;
  return SCGR_OK;
}
