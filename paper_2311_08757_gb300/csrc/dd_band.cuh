// Banded Cholesky solves, one warp per right-hand side, vector held in shared memory.
//
// Band storage of the lower factor L (half bandwidth b):
//   CB[i*(b+1) + d] = L(i+d, i)   (column band, used by the forward solve L y = r)
//   RB[i*(b+1) + d] = L(i, i-d)   (row band,    used by the backward solve L^T x = y)
//   inv[i]          = 1 / L(i, i)
// Both sweeps are written in "axpy" form: once x_i is known the lanes update the b
// entries it couples to, so each step costs one broadcast and b/32 FMAs per lane.
#pragma once

#include "dd_common.cuh"

namespace dd {

// Solves (L L^T) x = r in place in xs[0..n).  Caller: all 32 lanes of a warp, xs visible to
// the warp (shared memory), followed by __syncwarp() before xs is read elsewhere.
__device__ __forceinline__ void warp_band_solve(double* xs, int n, int b, const double* __restrict__ CB,
                                                const double* __restrict__ RB,
                                                const double* __restrict__ inv) {
  const int lane = threadIdx.x & 31;
  const int bs = b + 1;
  __syncwarp();
  for (int i = 0; i < n; ++i) {
    const double yi = xs[i] * __ldg(inv + i);
    const double* col = CB + (size_t)i * bs;
    const int dmax = min(b, n - 1 - i);
    for (int d = 1 + lane; d <= dmax; d += 32) xs[i + d] = fma(-__ldg(col + d), yi, xs[i + d]);
    __syncwarp();
    if (lane == 0) xs[i] = yi;
  }
  __syncwarp();
  for (int i = n - 1; i >= 0; --i) {
    const double xi = xs[i] * __ldg(inv + i);
    const double* row = RB + (size_t)i * bs;
    const int dmax = min(b, i);
    for (int d = 1 + lane; d <= dmax; d += 32) xs[i - d] = fma(-__ldg(row + d), xi, xs[i - d]);
    __syncwarp();
    if (lane == 0) xs[i] = xi;
  }
  __syncwarp();
}

}  // namespace dd
