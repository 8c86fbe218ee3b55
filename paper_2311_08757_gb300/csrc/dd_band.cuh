// Banded Cholesky solves, one warp per right-hand side, vector held in shared memory.
//
// Storage of the factor A = L L^T (half bandwidth b), pre-scaled by the pivots:
//   CB[i*(b+1) + d] = L(i+d, i) / L(i, i)       (column band; d = 0 unused)
//   RB[i*(b+1) + d] = L(i, i-d) / L(i-d, i-d)   (row band; RB[i][d] = CB[i-d][d])
//   inv[i]          = 1 / L(i, i)^2
// Forward sweep on w = L diag(L)^{-1}-scaled unknowns: w_{i+d} -= CB[i][d] w_i, then
// x_i = w_i inv_i, then the backward sweep x_{i-d} -= RB[i][d] x_i.  Every step is one
// broadcast of the pivot unknown and b/32 FMAs per lane, with no division or multiply on
// the sequential path.
#pragma once

#include "dd_common.cuh"

namespace dd {

// Solves (L L^T) x = r in place in xs[0..n).  Caller: all 32 lanes of a warp, xs visible to
// the warp (shared memory).
__device__ __forceinline__ void warp_band_solve(double* xs, int n, int b, const double* __restrict__ CB,
                                                const double* __restrict__ RB,
                                                const double* __restrict__ inv) {
  const int lane = threadIdx.x & 31;
  const int bs = b + 1;
  __syncwarp();
  for (int i = 0; i < n; ++i) {
    const double wi = xs[i];
    const double* col = CB + (size_t)i * bs;
    const int dmax = min(b, n - 1 - i);
    for (int d = 1 + lane; d <= dmax; d += 32) xs[i + d] = fma(-__ldg(col + d), wi, xs[i + d]);
    __syncwarp();
  }
  for (int i = lane; i < n; i += 32) xs[i] *= __ldg(inv + i);
  __syncwarp();
  for (int i = n - 1; i >= 0; --i) {
    const double xi = xs[i];
    const double* row = RB + (size_t)i * bs;
    const int dmax = min(b, i);
    for (int d = 1 + lane; d <= dmax; d += 32) xs[i - d] = fma(-__ldg(row + d), xi, xs[i - d]);
    __syncwarp();
  }
}

}  // namespace dd

namespace dd {

// Same solve with the band rows prefetched PF steps ahead into registers (a ring of PF
// rows, NV = ceil(b/32) values per lane), so the global-memory latency of the factor is
// off the sequential critical path.  The step loop is unrolled by PF so that the ring
// index is a compile-time constant.
template <int NV, int PF>
__device__ __forceinline__ void warp_band_solve_pf(double* xs, int n, int b, const double* __restrict__ CB,
                                                   const double* __restrict__ RB,
                                                   const double* __restrict__ inv) {
  const int lane = threadIdx.x & 31;
  const int bs = b + 1;
  double rb[PF][NV];
  // ---- forward sweep, rows 0, 1, ...
#pragma unroll
  for (int u = 0; u < PF; ++u) {
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      const int d = 1 + lane + 32 * v;
      rb[u][v] = (u < n && d <= b) ? __ldg(CB + (size_t)u * bs + d) : 0.0;
    }
  }
  __syncwarp();
  for (int i0 = 0; i0 < n; i0 += PF) {
#pragma unroll
    for (int u = 0; u < PF; ++u) {
      const int i = i0 + u;
      if (i < n) {
        const double wi = xs[i];
        const int dmax = min(b, n - 1 - i);
#pragma unroll
        for (int v = 0; v < NV; ++v) {
          const int d = 1 + lane + 32 * v;
          if (d <= dmax) xs[i + d] = fma(-rb[u][v], wi, xs[i + d]);
        }
        const int nx = i + PF;
#pragma unroll
        for (int v = 0; v < NV; ++v) {
          const int d = 1 + lane + 32 * v;
          rb[u][v] = (nx < n && d <= b) ? __ldg(CB + (size_t)nx * bs + d) : 0.0;
        }
        __syncwarp();
      }
    }
  }
  for (int i = lane; i < n; i += 32) xs[i] *= __ldg(inv + i);
  // ---- backward sweep, rows n-1, n-2, ...
#pragma unroll
  for (int u = 0; u < PF; ++u) {
    const int i = n - 1 - u;
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      const int d = 1 + lane + 32 * v;
      rb[u][v] = (i >= 0 && d <= b) ? __ldg(RB + (size_t)i * bs + d) : 0.0;
    }
  }
  __syncwarp();
  for (int i0 = 0; i0 < n; i0 += PF) {
#pragma unroll
    for (int u = 0; u < PF; ++u) {
      const int i = n - 1 - (i0 + u);
      if (i >= 0) {
        const double xi = xs[i];
        const int dmax = min(b, i);
#pragma unroll
        for (int v = 0; v < NV; ++v) {
          const int d = 1 + lane + 32 * v;
          if (d <= dmax) xs[i - d] = fma(-rb[u][v], xi, xs[i - d]);
        }
        const int nx = i - PF;
#pragma unroll
        for (int v = 0; v < NV; ++v) {
          const int d = 1 + lane + 32 * v;
          rb[u][v] = (nx >= 0 && d <= b) ? __ldg(RB + (size_t)nx * bs + d) : 0.0;
        }
        __syncwarp();
      }
    }
  }
}

// Host-side dispatch on the half bandwidth: BODY is compiled once per (NV, PF) pair.
#define DD_BAND_DISPATCH(b, BODY)                                   \
  do {                                                              \
    if ((b) <= 32) { constexpr int NV = 1, PF = 8; BODY; }          \
    else if ((b) <= 64) { constexpr int NV = 2, PF = 8; BODY; }     \
    else if ((b) <= 128) { constexpr int NV = 4, PF = 6; BODY; }    \
    else if ((b) <= 256) { constexpr int NV = 8, PF = 4; BODY; }    \
    else if ((b) <= 320) { constexpr int NV = 10, PF = 4; BODY; }   \
    else if ((b) <= 512) { constexpr int NV = 16, PF = 2; BODY; }   \
    else { constexpr int NV = 0, PF = 0; BODY; }                    \
  } while (0)

// NV = 0 selects the plain solve (bandwidths beyond 512)
template <int NV, int PF>
__device__ __forceinline__ void band_solve(double* xs, int n, int b, const double* __restrict__ CB,
                                           const double* __restrict__ RB, const double* __restrict__ inv) {
  if constexpr (NV == 0) warp_band_solve(xs, n, b, CB, RB, inv);
  else warp_band_solve_pf<NV, PF>(xs, n, b, CB, RB, inv);
}

}  // namespace dd
