// Exact k-nearest neighbours through a uniform grid, for large clouds.
//
// The result is identical to the brute-force search (reading R1): the same
// float32 key (dx*dx + dy*dy) + dz*dz without fused multiply-adds, the first
// k of the (key, index) order.  Points are counting-sorted into cells (the
// order inside a cell is arbitrary, so candidates are compared
// lexicographically by (key, index) rather than relying on scan order).  A
// query scans shells of cells around its own cell and stops once the k-th
// key is certified: every unscanned point lies at least dist_out from the
// query, where dist_out is the distance to the boundary of the scanned cube,
// and the float32 key of such a point exceeds dist_out^2 (1 - 1e-6) > k-th key.
#include <cfloat>
#include <climits>
#include <cmath>

#include "common.cuh"

namespace scgr {

constexpr int GRID_TPB = 128;

__global__ void minmax_kernel(const float4* __restrict__ P, int n, float* __restrict__ part) {
  __shared__ float sh[6][256];
  float lo[3] = {FLT_MAX, FLT_MAX, FLT_MAX}, hi[3] = {-FLT_MAX, -FLT_MAX, -FLT_MAX};
  for (int i = blockIdx.x * 256 + threadIdx.x; i < n; i += gridDim.x * 256) {
    const float4 c = P[i];
    lo[0] = fminf(lo[0], c.x); lo[1] = fminf(lo[1], c.y); lo[2] = fminf(lo[2], c.z);
    hi[0] = fmaxf(hi[0], c.x); hi[1] = fmaxf(hi[1], c.y); hi[2] = fmaxf(hi[2], c.z);
  }
  for (int a = 0; a < 3; ++a) {
    sh[a][threadIdx.x] = lo[a];
    sh[3 + a][threadIdx.x] = hi[a];
  }
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w)
      for (int a = 0; a < 3; ++a) {
        sh[a][threadIdx.x] = fminf(sh[a][threadIdx.x], sh[a][threadIdx.x + w]);
        sh[3 + a][threadIdx.x] = fmaxf(sh[3 + a][threadIdx.x], sh[3 + a][threadIdx.x + w]);
      }
    __syncthreads();
  }
  if (threadIdx.x == 0)
    for (int a = 0; a < 6; ++a) part[blockIdx.x * 6 + a] = sh[a][0];
}

__global__ void minmax_final_kernel(const float* __restrict__ part, int nb, float* __restrict__ out) {
  if (threadIdx.x != 0) return;
  float r[6] = {FLT_MAX, FLT_MAX, FLT_MAX, -FLT_MAX, -FLT_MAX, -FLT_MAX};
  for (int b = 0; b < nb; ++b)
    for (int a = 0; a < 3; ++a) {
      r[a] = fminf(r[a], part[b * 6 + a]);
      r[3 + a] = fmaxf(r[3 + a], part[b * 6 + 3 + a]);
    }
  for (int a = 0; a < 6; ++a) out[a] = r[a];
}

__device__ __forceinline__ int cell_coord(float v, double o, double inv_h, int g) {
  int c = (int)floor(((double)v - o) * inv_h);
  return c < 0 ? 0 : (c >= g ? g - 1 : c);
}

__global__ void cell_count_kernel(const float4* __restrict__ P, int n, GridSpec gs, int* __restrict__ cell_of,
                                  int* __restrict__ count) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float4 c = P[i];
  const int cx = cell_coord(c.x, gs.o[0], gs.inv_h, gs.g[0]);
  const int cy = cell_coord(c.y, gs.o[1], gs.inv_h, gs.g[1]);
  const int cz = cell_coord(c.z, gs.o[2], gs.inv_h, gs.g[2]);
  const int cell = (cz * gs.g[1] + cy) * gs.g[0] + cx;
  cell_of[i] = cell;
  atomicAdd(count + cell, 1);
}

// Exclusive scan of count[0, ncell) into start[0, ncell] (start[ncell] = n),
// in three passes over blocks of 1024 cells.
constexpr int SCAN_B = 1024;

__global__ void scan_local_kernel(const int* __restrict__ count, int ncell, int* __restrict__ start,
                                  int* __restrict__ block_tot) {
  __shared__ int sh[SCAN_B];
  const int base = blockIdx.x * SCAN_B;
  for (int t = threadIdx.x; t < SCAN_B; t += blockDim.x) sh[t] = (base + t < ncell) ? count[base + t] : 0;
  __syncthreads();
  if (threadIdx.x == 0) {
    int run = 0;
    for (int t = 0; t < SCAN_B; ++t) {
      const int v = sh[t];
      sh[t] = run;
      run += v;
    }
    block_tot[blockIdx.x] = run;
  }
  __syncthreads();
  for (int t = threadIdx.x; t < SCAN_B; t += blockDim.x)
    if (base + t < ncell) start[base + t] = sh[t];
}

__global__ void scan_blocks_kernel(int* __restrict__ block_tot, int nblocks, int* __restrict__ start, int ncell) {
  if (threadIdx.x != 0) return;
  int run = 0;
  for (int b = 0; b < nblocks; ++b) {
    const int v = block_tot[b];
    block_tot[b] = run;
    run += v;
  }
  start[ncell] = run;
}

__global__ void scan_add_kernel(int* __restrict__ start, int ncell, const int* __restrict__ block_tot) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < ncell) start[i] += block_tot[i / SCAN_B];
}

__global__ void scatter_kernel(const float4* __restrict__ P, int n, const int* __restrict__ cell_of,
                               const int* __restrict__ start, int* __restrict__ cursor, float4* __restrict__ sorted,
                               int* __restrict__ sorted_idx) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int cell = cell_of[i];
  const int pos = start[cell] + atomicAdd(cursor + cell, 1);
  sorted[pos] = P[i];
  sorted_idx[pos] = i;
}

__device__ __forceinline__ bool lex_less(float ka, int ia, float kb, int ib) {
  return ka < kb || (ka == kb && ia < ib);
}

// The k (<= KC) first (key, index) neighbours of query q among the gridded
// points: shells of cells around q's cell (clamped to the grid, so q may lie
// outside the box), stopping once the k-th key is certified.  Every point
// not yet scanned lies beyond a face of the scanned cube that has grid cells
// behind it, and q is on the inner side of each such face, so its distance
// to q is at least the distance dist_out from q to the nearest such face.
template <int KC>
__device__ __forceinline__ void grid_scan(const float4 q, const float4* __restrict__ sorted,
                                          const int* __restrict__ sorted_idx, const int* __restrict__ start,
                                          int k, const GridSpec& gs, float (&kd)[KC], int (&ki)[KC]) {
  const int cx = cell_coord(q.x, gs.o[0], gs.inv_h, gs.g[0]);
  const int cy = cell_coord(q.y, gs.o[1], gs.inv_h, gs.g[1]);
  const int cz = cell_coord(q.z, gs.o[2], gs.inv_h, gs.g[2]);
#pragma unroll
  for (int m = 0; m < KC; ++m) {
    kd[m] = INFINITY;
    ki[m] = INT_MAX;
  }
  const int smax = max(gs.g[0], max(gs.g[1], gs.g[2]));
  for (int s = 0; s <= smax; ++s) {
    for (int dz = -s; dz <= s; ++dz) {
      const int z = cz + dz;
      if (z < 0 || z >= gs.g[2]) continue;
      for (int dy = -s; dy <= s; ++dy) {
        const int y = cy + dy;
        if (y < 0 || y >= gs.g[1]) continue;
        const bool face = (dz == -s || dz == s || dy == -s || dy == s);
        const int step = face ? 1 : (s > 0 ? 2 * s : 1);
        for (int dx = -s; dx <= s; dx += step) {
          const int x = cx + dx;
          if (x < 0 || x >= gs.g[0]) continue;
          const int cell = (z * gs.g[1] + y) * gs.g[0] + x;
          const int e = start[cell + 1];
          for (int j = start[cell]; j < e; ++j) {
            const float4 c = sorted[j];
            const float ex = __fsub_rn(q.x, c.x);
            const float ey = __fsub_rn(q.y, c.y);
            const float ez = __fsub_rn(q.z, c.z);
            const float key = __fadd_rn(__fadd_rn(__fmul_rn(ex, ex), __fmul_rn(ey, ey)), __fmul_rn(ez, ez));
            const int idx = sorted_idx[j];
            if (lex_less(key, idx, kd[KC - 1], ki[KC - 1])) {
              kd[KC - 1] = key;
              ki[KC - 1] = idx;
#pragma unroll
              for (int m = KC - 1; m > 0; --m) {
                if (lex_less(kd[m], ki[m], kd[m - 1], ki[m - 1])) {
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
        }
      }
    }
    // distance from q to the outside of the scanned cube of cells; a side on
    // the grid boundary has nothing beyond it
    double dout = INFINITY;
    const int cc[3] = {cx, cy, cz};
    const float qq[3] = {q.x, q.y, q.z};
    bool all = true;
    for (int a = 0; a < 3; ++a) {
      if (cc[a] - s > 0) {
        dout = fmin(dout, (double)qq[a] - (gs.o[a] + (double)(cc[a] - s) * gs.h));
        all = false;
      }
      if (cc[a] + s < gs.g[a] - 1) {
        dout = fmin(dout, (gs.o[a] + (double)(cc[a] + s + 1) * gs.h) - (double)qq[a]);
        all = false;
      }
    }
    if (all) break;
    const int kk = k < KC ? k : KC;
    if (ki[kk - 1] != INT_MAX && dout > 0.0 && (double)kd[kk - 1] < dout * dout * (1.0 - 1e-6)) break;
  }
}

// k nearest neighbours of every point of the gridded cloud itself.
template <int KC>
__global__ void __launch_bounds__(GRID_TPB)
    knn_grid_query_kernel(const float4* __restrict__ sorted, const int* __restrict__ sorted_idx,
                          const int* __restrict__ start, int n, int k, GridSpec gs, int32_t* __restrict__ out) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  const float4 q = sorted[t];  // queries in cell order: neighbouring threads share cells
  const int qi = sorted_idx[t];
  float kd[KC];
  int ki[KC];
  grid_scan<KC>(q, sorted, sorted_idx, start, k, gs, kd, ki);
#pragma unroll
  for (int m = 0; m < KC; ++m)
    if (m < k) out[(int64_t)qi * k + m] = ki[m];
}

// Nearest gridded point (first of the (key, index) order) of each of nq
// external queries q3 [nq][3] (float32); key = the float32 squared distance.
__global__ void __launch_bounds__(GRID_TPB)
    nearest_grid_kernel(const float4* __restrict__ sorted, const int* __restrict__ sorted_idx,
                        const int* __restrict__ start, GridSpec gs, const float* __restrict__ q3, int nq,
                        int32_t* __restrict__ idx_out, float* __restrict__ key_out) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nq) return;
  const float4 q = make_float4(q3[3 * (size_t)t], q3[3 * (size_t)t + 1], q3[3 * (size_t)t + 2], 0.f);
  float kd[1];
  int ki[1];
  grid_scan<1>(q, sorted, sorted_idx, start, 1, gs, kd, ki);
  if (idx_out) idx_out[t] = ki[0];
  if (key_out) key_out[t] = kd[0];
}

// Nearest gridded point (k = 1, first of the (key, index) order) over the
// shells 0..smax of cells around q's cell in grid g.  With `prune`, a
// non-empty cell is skipped when every point of its box is farther than the
// best key so far (its squared box distance, less a 1e-6 margin for the
// rounding of the float32 key, exceeds that key, so no point in it can even
// tie).  Re-scanning a point already seen leaves the best unchanged.
// Returns true once the best is certified by the stop rule of grid_scan (or
// the whole grid has been scanned).
__device__ __forceinline__ bool nearest_shells(const float4 q, const float4* __restrict__ sorted,
                                               const int* __restrict__ sorted_idx, const int* __restrict__ start,
                                               const GridSpec& g, int smax, bool prune, float& bk, int& bi) {
  const int cc[3] = {cell_coord(q.x, g.o[0], g.inv_h, g.g[0]), cell_coord(q.y, g.o[1], g.inv_h, g.g[1]),
                     cell_coord(q.z, g.o[2], g.inv_h, g.g[2])};
  const float qq[3] = {q.x, q.y, q.z};
  const int sgrid = max(g.g[0], max(g.g[1], g.g[2]));
  const int slast = smax < sgrid ? smax : sgrid;
  for (int s = 0; s <= slast; ++s) {
    for (int dz = -s; dz <= s; ++dz) {
      const int z = cc[2] + dz;
      if (z < 0 || z >= g.g[2]) continue;
      for (int dy = -s; dy <= s; ++dy) {
        const int y = cc[1] + dy;
        if (y < 0 || y >= g.g[1]) continue;
        const bool face = (dz == -s || dz == s || dy == -s || dy == s);
        const int step = face ? 1 : (s > 0 ? 2 * s : 1);
        for (int dx = -s; dx <= s; dx += step) {
          const int x = cc[0] + dx;
          if (x < 0 || x >= g.g[0]) continue;
          const int cell = (z * g.g[1] + y) * g.g[0] + x;
          const int b = start[cell], e = start[cell + 1];
          if (b == e) continue;
          if (prune && bi != INT_MAX) {
            const int xyz[3] = {x, y, z};
            double d2 = 0.0;
            for (int a = 0; a < 3; ++a) {
              const double lo = g.o[a] + (double)xyz[a] * g.h;
              const double hi = lo + g.h;
              const double v = (double)qq[a];
              const double d = v < lo ? lo - v : (v > hi ? v - hi : 0.0);
              d2 += d * d;
            }
            if (d2 * (1.0 - 1e-6) > (double)bk) continue;
          }
          for (int j = b; j < e; ++j) {
            const float4 c = sorted[j];
            const float ex = __fsub_rn(q.x, c.x);
            const float ey = __fsub_rn(q.y, c.y);
            const float ez = __fsub_rn(q.z, c.z);
            const float key = __fadd_rn(__fadd_rn(__fmul_rn(ex, ex), __fmul_rn(ey, ey)), __fmul_rn(ez, ez));
            const int idx = sorted_idx[j];
            if (lex_less(key, idx, bk, bi)) {
              bk = key;
              bi = idx;
            }
          }
        }
      }
    }
    double dout = INFINITY;
    bool all = true;
    for (int a = 0; a < 3; ++a) {
      if (cc[a] - s > 0) {
        dout = fmin(dout, (double)qq[a] - (g.o[a] + (double)(cc[a] - s) * g.h));
        all = false;
      }
      if (cc[a] + s < g.g[a] - 1) {
        dout = fmin(dout, (g.o[a] + (double)(cc[a] + s + 1) * g.h) - (double)qq[a]);
        all = false;
      }
    }
    if (all) return true;
    if (bi != INT_MAX && dout > 0.0 && (double)bk < dout * dout * (1.0 - 1e-6)) return true;
  }
  return false;
}

// Two-level exact nearest search: the query's own cell and its neighbours
// in the fine grid (enough for a query on the surface), then, if that does
// not certify the nearest point, shells of the coarse grid (cells of
// NEAREST_COARSE fine cells a side, points sorted by coarse cell) that skip
// empty coarse cells and coarse cells beyond the best key.  A query far off
// the surface then visits a few hundred coarse cells instead of the
// (1.7 D / h)^3 fine cells a fine shell scan needs to certify distance D.
// The result is the (key, index)-first point, as the one-level search gives.
__global__ void __launch_bounds__(GRID_TPB)
    nearest_grid2_kernel(const float4* __restrict__ sorted, const int* __restrict__ sorted_idx,
                         const int* __restrict__ start, GridSpec gs, const float4* __restrict__ csorted,
                         const int* __restrict__ csorted_idx, const int* __restrict__ cstart, GridSpec gc,
                         const float* __restrict__ q3, int nq, int32_t* __restrict__ idx_out,
                         float* __restrict__ key_out) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nq) return;
  const float4 q = make_float4(q3[3 * (size_t)t], q3[3 * (size_t)t + 1], q3[3 * (size_t)t + 2], 0.f);
  float bk = INFINITY;
  int bi = INT_MAX;
  if (!nearest_shells(q, sorted, sorted_idx, start, gs, 1, false, bk, bi))
    nearest_shells(q, csorted, csorted_idx, cstart, gc, INT_MAX, true, bk, bi);
  if (idx_out) idx_out[t] = bi;
  if (key_out) key_out[t] = bk;
}

// The coarse grid over the same origin: cells of NEAREST_COARSE fine cells a side.
GridSpec coarse_grid_spec(const GridSpec& gs) {
  GridSpec gc = gs;
  gc.h = gs.h * NEAREST_COARSE;
  gc.inv_h = 1.0 / gc.h;
  for (int a = 0; a < 3; ++a) gc.g[a] = (gs.g[a] + NEAREST_COARSE - 1) / NEAREST_COARSE;
  return gc;
}

cudaError_t launch_nearest_grid2(Launch L, const float4* sorted, const int* sorted_idx, const int* start,
                                 const GridSpec& gs, const float4* csorted, const int* csorted_idx,
                                 const int* cstart, const GridSpec& gc, const float* q3, int nq, int32_t* idx_out,
                                 float* key_out) {
  if (nq <= 0) return cudaSuccess;
  nearest_grid2_kernel<<<(nq + GRID_TPB - 1) / GRID_TPB, GRID_TPB, 0, L.stream>>>(
      sorted, sorted_idx, start, gs, csorted, csorted_idx, cstart, gc, q3, nq, idx_out, key_out);
  if (L.counter) *L.counter += 1;
  return cudaGetLastError();
}

// Grid spec from the bounding box: cell edge h = sqrt(8 A / n) with A the box
// surface area (about 8 points per occupied cell on a surface sample), at most
// 8 n cells, at least one cell per axis.
GridSpec make_grid_spec(const float* bb, int64_t n) {
  GridSpec gs;
  double e[3];
  for (int a = 0; a < 3; ++a) e[a] = (double)bb[3 + a] - (double)bb[a];
  const double A = 2.0 * (e[0] * e[1] + e[1] * e[2] + e[2] * e[0]);
  const double emax = fmax(e[0], fmax(e[1], e[2]));
  double h = A > 0.0 ? sqrt(8.0 * A / (double)n) : (emax > 0.0 ? emax * 8.0 / (double)n : 1.0);
  if (!(h > 0.0)) h = 1.0;
  for (int it = 0; it < 64; ++it) {
    double cells = 1.0;
    for (int a = 0; a < 3; ++a) cells *= fmax(1.0, ceil(e[a] / h + 1e-9));
    if (cells <= 8.0 * (double)n + 8.0) break;
    h *= 1.25;
  }
  gs.h = h;
  gs.inv_h = 1.0 / h;
  for (int a = 0; a < 3; ++a) {
    gs.o[a] = (double)bb[a];
    gs.g[a] = (int)fmax(1.0, ceil(e[a] / h + 1e-9));
  }
  return gs;
}

int64_t grid_cells(const GridSpec& gs) { return (int64_t)gs.g[0] * gs.g[1] * gs.g[2]; }

cudaError_t launch_bbox(Launch L, const float4* P, int n, float* part, float* out6) {
  const int nb = 256;
  minmax_kernel<<<nb, 256, 0, L.stream>>>(P, n, part);
  minmax_final_kernel<<<1, 32, 0, L.stream>>>(part, nb, out6);
  if (L.counter) *L.counter += 2;
  return cudaGetLastError();
}

// Counting sort of the n points into the cells of gs: sorted / sorted_idx in
// cell order, start[ncell + 1] the cell offsets.
cudaError_t launch_grid_build(Launch L, const float4* P, int n, const GridSpec& gs, int* cell_of, int* count,
                              int* start, int* cursor, int* block_tot, float4* sorted, int* sorted_idx) {
  const int64_t ncell = grid_cells(gs);
  cudaError_t e = cudaMemsetAsync(count, 0, (size_t)ncell * sizeof(int), L.stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(cursor, 0, (size_t)ncell * sizeof(int), L.stream);
  if (e != cudaSuccess) return e;
  const int tpb = 256;
  cell_count_kernel<<<(n + tpb - 1) / tpb, tpb, 0, L.stream>>>(P, n, gs, cell_of, count);
  const int nsb = (int)((ncell + SCAN_B - 1) / SCAN_B);
  scan_local_kernel<<<nsb, 256, 0, L.stream>>>(count, (int)ncell, start, block_tot);
  scan_blocks_kernel<<<1, 32, 0, L.stream>>>(block_tot, nsb, start, (int)ncell);
  scan_add_kernel<<<(int)((ncell + tpb - 1) / tpb), tpb, 0, L.stream>>>(start, (int)ncell, block_tot);
  scatter_kernel<<<(n + tpb - 1) / tpb, tpb, 0, L.stream>>>(P, n, cell_of, start, cursor, sorted, sorted_idx);
  if (L.counter) *L.counter += 5;
  return cudaGetLastError();
}

cudaError_t launch_knn_grid(Launch L, const float4* P, int n, int k, const GridSpec& gs, int* cell_of, int* count,
                            int* start, int* cursor, int* block_tot, float4* sorted, int* sorted_idx,
                            int32_t* out) {
  cudaError_t e = launch_grid_build(L, P, n, gs, cell_of, count, start, cursor, block_tot, sorted, sorted_idx);
  if (e != cudaSuccess) return e;
  const unsigned qb = (unsigned)((n + GRID_TPB - 1) / GRID_TPB);
  if (k <= 8) knn_grid_query_kernel<8><<<qb, GRID_TPB, 0, L.stream>>>(sorted, sorted_idx, start, n, k, gs, out);
  else if (k <= 16) knn_grid_query_kernel<16><<<qb, GRID_TPB, 0, L.stream>>>(sorted, sorted_idx, start, n, k, gs, out);
  else knn_grid_query_kernel<32><<<qb, GRID_TPB, 0, L.stream>>>(sorted, sorted_idx, start, n, k, gs, out);
  if (L.counter) *L.counter += 1;
  return cudaGetLastError();
}

cudaError_t launch_nearest_grid(Launch L, const float4* sorted, const int* sorted_idx, const int* start,
                                const GridSpec& gs, const float* q3, int nq, int32_t* idx_out, float* key_out) {
  if (nq <= 0) return cudaSuccess;
  nearest_grid_kernel<<<(nq + GRID_TPB - 1) / GRID_TPB, GRID_TPB, 0, L.stream>>>(sorted, sorted_idx, start, gs, q3,
                                                                                nq, idx_out, key_out);
  if (L.counter) *L.counter += 1;
  return cudaGetLastError();
}

}  // namespace scgr
