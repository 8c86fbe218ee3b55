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

__device__ __forceinline__ double fma_el(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ float fma_el(float a, float b, float c) { return fmaf(a, b, c); }

// Solves (L L^T) x = r in place in xs[0..n).  Caller: all 32 lanes of a warp, xs visible to
// the warp (shared memory).  T is double (the plain method, the coarse factor) or float (the
// factors whose inverses are rounded to a tensor-core type, and the cell preconditioner).
template <typename T>
__device__ __forceinline__ void warp_band_solve(T* xs, int n, int b, const T* __restrict__ CB,
                                                const T* __restrict__ RB, const T* __restrict__ inv) {
  const int lane = threadIdx.x & 31;
  const int bs = b + 1;
  __syncwarp();
  for (int i = 0; i < n; ++i) {
    const T wi = xs[i];
    const T* col = CB + (size_t)i * bs;
    const int dmax = min(b, n - 1 - i);
    for (int d = 1 + lane; d <= dmax; d += 32) xs[i + d] = fma_el(-__ldg(col + d), wi, xs[i + d]);
    __syncwarp();
  }
  for (int i = lane; i < n; i += 32) xs[i] *= __ldg(inv + i);
  __syncwarp();
  for (int i = n - 1; i >= 0; --i) {
    const T xi = xs[i];
    const T* row = RB + (size_t)i * bs;
    const int dmax = min(b, i);
    for (int d = 1 + lane; d <= dmax; d += 32) xs[i - d] = fma_el(-__ldg(row + d), xi, xs[i - d]);
    __syncwarp();
  }
}

}  // namespace dd

namespace dd {

// Host-side dispatch on the half bandwidth: BODY is compiled once per (NV, PF) pair.
#define DD_BAND_DISPATCH(b, BODY)                                   \
  do {                                                              \
    if ((b) <= 32) { constexpr int NV = 1, PF = 24; BODY; }         \
    else if ((b) <= 64) { constexpr int NV = 2, PF = 16; BODY; }    \
    else if ((b) <= 128) { constexpr int NV = 4, PF = 6; BODY; }    \
    else if ((b) <= 256) { constexpr int NV = 8, PF = 4; BODY; }    \
    else if ((b) <= 320) { constexpr int NV = 10, PF = 4; BODY; }   \
    else if ((b) <= 512) { constexpr int NV = 16, PF = 2; BODY; }   \
    else { constexpr int NV = 0, PF = 0; BODY; }                    \
  } while (0)

}  // namespace dd

namespace dd {

// Asynchronous 8- or 4-byte global -> shared copies (cp.async), committed one group per band row.
__device__ __forceinline__ void cp_async_el(double* dst_smem, const double* src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst_smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_el(float* dst_smem, const float* src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst_smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// shared-memory ring of the band-coefficient prefetch: PF rows x NV values x 32 lanes
// (elements of the factor's type)
template <int NV, int PF>
__host__ __device__ constexpr int band_ring_elems() { return NV > 0 ? PF * NV * 32 : 0; }

// Lane-owned solve of K right-hand sides sharing one factor (vector k at xs + k * ldx).
// Element j of every vector belongs to lane j & 31 for the whole solve: each lane keeps its
// elements of the active band window in registers (e[t] = element jlo + 32 t, jlo its
// lowest element not yet past the pivot) and reads and writes only its own shared-memory
// slots, so no warp barrier sits on the sequential path.  The only exchange per step is the
// broadcast of the pivot value by its owner lane (shuffle):
//   forward, i = 0..n-1:  w_i from lane i&31;  e[t] -= CB[i][d_t] w_i for the lane's
//                         elements j = i + d_t in the band, d_t = ((lane - i - 1) & 31) + 1 + 32 t;
//   scale:                x_j = w_j inv_j (own elements);
//   backward, i = n-1..0: x_i from lane i&31;  e[t] -= RB[i][d_t] x_i for j = i - d_t,
//                         d_t = ((i - lane - 1) & 31) + 1 + 32 t.
// The owner of the pivot stores it to its slot and shifts its window by one element; the
// element entering the window is an untouched value of its own slot, loaded 32 steps early.
// The band coefficients of row i + PF are copied asynchronously (cp.async, one commit
// group per row) into this lane's slot of a PF-row ring while row i is used: a wait on the
// group count keeps PF rows in flight, which register prefetches cannot (their completion
// is tracked by a handful of scoreboards, so a use waits on recent loads too).  Each lane
// reads back only the slots it copied itself.  Per vector the floating-point operations are
// those of warp_band_solve, in the same order, so the results are identical.
template <int NV, int PF, int K, typename T>
__device__ __forceinline__ void warp_band_solve_k(T* xs, int ldx, int n, int b, const T* __restrict__ CB,
                                                  const T* __restrict__ RB, const T* __restrict__ inv, T* ring) {
  const int lane = threadIdx.x & 31;
  const int bs = b + 1;
  T e[K][NV], nx[K];
  T* rl = ring + lane;   // this lane's column of the ring: slot (u, t) at rl[(u * NV + t) * 32]
  // ---- forward sweep
#pragma unroll
  for (int k = 0; k < K; ++k) {
#pragma unroll
    for (int t = 0; t < NV; ++t) e[k][t] = xs[k * ldx + min(lane + 32 * t, n - 1)];
    nx[k] = xs[k * ldx + min(lane + 32 * NV, n - 1)];
  }
#pragma unroll
  for (int u = 0; u < PF; ++u) {
#pragma unroll
    for (int t = 0; t < NV; ++t) {
      const int d = ((lane - u - 1) & 31) + 1 + 32 * t;
      cp_async_el(rl + (u * NV + t) * 32, CB + (size_t)min(u, n - 1) * bs + min(d, b));
    }
    cp_async_commit();
  }
  for (int i0 = 0; i0 < n; i0 += PF) {
#pragma unroll
    for (int u = 0; u < PF; ++u) {
      const int i = i0 + u;
      if (i < n) {
        cp_async_wait<PF - 1>();
        T rb[NV];
#pragma unroll
        for (int t = 0; t < NV; ++t) rb[t] = rl[(u * NV + t) * 32];
        const int piv = i & 31;
        T w[K];
#pragma unroll
        for (int k = 0; k < K; ++k) w[k] = __shfl_sync(kFull, e[k][0], piv);
        if (lane == piv) {
#pragma unroll
          for (int k = 0; k < K; ++k) {
            xs[k * ldx + i] = w[k];
#pragma unroll
            for (int t = 0; t < NV - 1; ++t) e[k][t] = e[k][t + 1];
            e[k][NV - 1] = nx[k];
            nx[k] = xs[k * ldx + min(i + 32 + 32 * NV, n - 1)];
          }
        }
#pragma unroll
        for (int t = 0; t < NV; ++t) {
          const int d = ((lane - i - 1) & 31) + 1 + 32 * t;
          if (d <= b && i + d < n) {
#pragma unroll
            for (int k = 0; k < K; ++k) e[k][t] = fma_el(-rb[t], w[k], e[k][t]);
          }
        }
        const int ni = i + PF;
#pragma unroll
        for (int t = 0; t < NV; ++t) {
          const int d = ((lane - ni - 1) & 31) + 1 + 32 * t;
          cp_async_el(rl + (u * NV + t) * 32, CB + (size_t)min(ni, n - 1) * bs + min(d, b));
        }
        cp_async_commit();
      }
    }
  }
  cp_async_wait<0>();
  // ---- scale by 1 / L_jj^2 (own elements)
  for (int j = lane; j < n; j += 32) {
    const T sc = __ldg(inv + j);
#pragma unroll
    for (int k = 0; k < K; ++k) xs[k * ldx + j] *= sc;
  }
  // ---- backward sweep: e[t] = element jhi - 32 t, jhi the lane's highest element <= i
  const int jhi = (n - 1) - ((n - 1 - lane) & 31);
#pragma unroll
  for (int k = 0; k < K; ++k) {
#pragma unroll
    for (int t = 0; t < NV; ++t) e[k][t] = xs[k * ldx + max(jhi - 32 * t, 0)];
    nx[k] = xs[k * ldx + max(jhi - 32 * NV, 0)];
  }
#pragma unroll
  for (int u = 0; u < PF; ++u) {
    const int i = n - 1 - u;
#pragma unroll
    for (int t = 0; t < NV; ++t) {
      const int d = ((i - lane - 1) & 31) + 1 + 32 * t;
      cp_async_el(rl + (u * NV + t) * 32, RB + (size_t)max(i, 0) * bs + min(d, b));
    }
    cp_async_commit();
  }
  for (int i0 = 0; i0 < n; i0 += PF) {
#pragma unroll
    for (int u = 0; u < PF; ++u) {
      const int i = n - 1 - (i0 + u);
      if (i >= 0) {
        cp_async_wait<PF - 1>();
        T rb[NV];
#pragma unroll
        for (int t = 0; t < NV; ++t) rb[t] = rl[(u * NV + t) * 32];
        const int piv = i & 31;
        T xv[K];
#pragma unroll
        for (int k = 0; k < K; ++k) xv[k] = __shfl_sync(kFull, e[k][0], piv);
        if (lane == piv) {
#pragma unroll
          for (int k = 0; k < K; ++k) {
            xs[k * ldx + i] = xv[k];
#pragma unroll
            for (int t = 0; t < NV - 1; ++t) e[k][t] = e[k][t + 1];
            e[k][NV - 1] = nx[k];
            nx[k] = xs[k * ldx + max(i - 32 - 32 * NV, 0)];
          }
        }
#pragma unroll
        for (int t = 0; t < NV; ++t) {
          const int d = ((i - lane - 1) & 31) + 1 + 32 * t;
          if (d <= b && i - d >= 0) {
#pragma unroll
            for (int k = 0; k < K; ++k) e[k][t] = fma_el(-rb[t], xv[k], e[k][t]);
          }
        }
        const int ni = i - PF;
#pragma unroll
        for (int t = 0; t < NV; ++t) {
          const int d = ((ni - lane - 1) & 31) + 1 + 32 * t;
          cp_async_el(rl + (u * NV + t) * 32, RB + (size_t)max(ni, 0) * bs + min(d, b));
        }
        cp_async_commit();
      }
    }
  }
  cp_async_wait<0>();
}

// K-way solve for NV > 0; the plain single-vector solve otherwise (K = 1 then)
template <int NV, int PF, int K, typename T>
__device__ __forceinline__ void band_solve_k(T* xs, int ldx, int n, int b, const T* __restrict__ CB,
                                             const T* __restrict__ RB, const T* __restrict__ inv, T* ring) {
  if constexpr (NV == 0) warp_band_solve(xs, n, b, CB, RB, inv);
  else warp_band_solve_k<NV, PF, K>(xs, ldx, n, b, CB, RB, inv, ring);
}

// bytes of the coefficient ring per warp for half bandwidth b and element size es (host side)
inline size_t band_ring_bytes(int b, size_t es = sizeof(double)) {
  size_t r = 0;
  DD_BAND_DISPATCH(b, (r = es * (size_t)band_ring_elems<NV, PF>()));
  return r;
}

// largest number of right-hand sides per warp for local vectors of n_max doubles (shared
// memory per warp); the local solves use two where allowed (measured fastest at h = 1/32)
inline int rhs_per_warp(int nmax, int b) {
  if (b > 128) return 1;   // wide bands: one vector per warp (registers)
  const size_t per = (size_t)nmax * sizeof(double);
  if (4 * per <= 48 * 1024) return 4;
  if (2 * per <= 64 * 1024) return 2;
  return 1;
}

#define DD_K_DISPATCH(k, BODY)                              \
  do {                                                      \
    if ((k) == 4) { constexpr int KR = 4; BODY; }           \
    else if ((k) == 2) { constexpr int KR = 2; BODY; }      \
    else { constexpr int KR = 1; BODY; }                    \
  } while (0)

}  // namespace dd
