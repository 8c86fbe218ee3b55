// Rayleigh-Ritz step on a three-vector search space from its Gram matrices (Algorithm 1),
// shared by the SI-LOPCG outer step and the cell eigen-solve.
#pragma once

#include "dd_common.cuh"

namespace dd {

// index of the upper-triangular entry (i, j), i <= j, of a symmetric 3 x 3 matrix
__device__ __forceinline__ int sym3(int i, int j) {
  if (i > j) {
    const int t = i;
    i = j;
    j = t;
  }
  return i == 0 ? j : (i == 1 ? 2 + j : 5);
}

// Everything below indexes its 3 x 3 arrays with compile-time indices only (fully unrolled),
// so they stay in registers: runtime indexing put them in local memory, and every dependent
// step paid a memory round trip on top of GB300's 64-cycle FP64 latency.

// One Jacobi rotation in the (p, q) plane: H <- J^T H J, V <- V J.  The angle (t = tan phi,
// tau = cot 2 phi) is formed in FP32: GB300's FP64 divide and square root are long dependent
// chains on one thread; normalising (cs, sn) in FP64 keeps the rotation orthogonal to FP64
// rounding, and an angle good to FP32 still cuts H[p][q] by about 1e-7, so the sweeps end as
// with exact angles.
template <int p, int q>
__device__ __forceinline__ void jacobi_rotate(double (&H)[3][3], double (&V)[3][3]) {
  const double hpq = H[p][q];
  if (hpq == 0.0) return;
  const double dq = H[q][q] - H[p][p];
  double t;
  const float fp = (float)hpq, fd = (float)dq;
  if (fabsf(fp) > 1e-30f && fabsf(fp) < 1e30f && fabsf(fd) < 1e30f) {
    const float tau = fd / (2.0f * fp);
    t = (double)(copysignf(1.0f, tau) / (fabsf(tau) + sqrtf(fmaf(tau, tau, 1.0f))));
  } else {
    const double tau = dq / (2.0 * hpq);
    t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
  }
  const double cs = rsqrt(fma(t, t, 1.0)), sn = t * cs;
#pragma unroll
  for (int k = 0; k < 3; ++k) {   // H <- H J
    const double hp = H[k][p], hq = H[k][q];
    H[k][p] = cs * hp - sn * hq;
    H[k][q] = sn * hp + cs * hq;
  }
#pragma unroll
  for (int k = 0; k < 3; ++k) {   // H <- J^T H
    const double hp = H[p][k], hq = H[q][k];
    H[p][k] = cs * hp - sn * hq;
    H[q][k] = sn * hp + cs * hq;
  }
#pragma unroll
  for (int k = 0; k < 3; ++k) {   // V <- V J
    const double vp = V[k][p], vq = V[k][q];
    V[k][p] = cs * vp - sn * vq;
    V[k][q] = sn * vp + cs * vq;
  }
}

// Lowest eigenpair of the symmetric 3 x 3 matrix H by cyclic Jacobi sweeps (symmetric Schur
// decompositions of 2 x 2 blocks), until the off-diagonal mass is below the rounding of the
// diagonal.
__device__ inline void jacobi_lowest(double (&H)[3][3], double* theta, double (&y)[3]) {
  double V[3][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}};
#pragma unroll 1
  for (int sweep = 0; sweep < 50; ++sweep) {
    const double off = H[0][1] * H[0][1] + H[0][2] * H[0][2] + H[1][2] * H[1][2];
    const double dia = H[0][0] * H[0][0] + H[1][1] * H[1][1] + H[2][2] * H[2][2];
    if (off <= 1e-34 * dia) break;
    jacobi_rotate<0, 1>(H, V);
    jacobi_rotate<0, 2>(H, V);
    jacobi_rotate<1, 2>(H, V);
  }
  const int lo = (H[0][0] <= H[1][1]) ? ((H[0][0] <= H[2][2]) ? 0 : 2) : ((H[1][1] <= H[2][2]) ? 1 : 2);
  *theta = (lo == 0) ? H[0][0] : ((lo == 1) ? H[1][1] : H[2][2]);
#pragma unroll
  for (int k = 0; k < 3; ++k) y[k] = (lo == 0) ? V[k][0] : ((lo == 1) ? V[k][1] : V[k][2]);
}

// Orthogonalised Rayleigh-Ritz on span{x_k, w_k, x_{k-1}} from the Gram matrices (Algorithm 1):
// Gram-Schmidt in the M inner product on coefficient vectors (order x_k, w_k, x_{k-1}, two
// passes; a direction whose M-norm falls to drop times its norm before is dropped: its column
// stays zero), lowest eigenpair of the projected matrix (a dropped direction gets a decoupled
// diagonal entry above all others), coefficients signed so that the sum of the Ritz vector is
// positive.
__device__ inline void rayleigh_ritz3(LopState* ls, double drop) {
  double GA[3][3], GB[3][3];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      GA[i][j] = ls->GA[sym3(i, j)];
      GB[i][j] = ls->GB[sym3(i, j)];
    }
  double T[3][3];   // columns: accepted coefficient vectors (zero when dropped)
  bool acc[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    double v[3] = {0.0, 0.0, 0.0};
    v[i] = 1.0;
    const double n0 = GB[i][i];
#pragma unroll
    for (int pass = 0; pass < 2; ++pass)
#pragma unroll
      for (int k = 0; k < i; ++k) {   // dropped columns are zero: their projection is zero
        double gv[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) gv[a] = GB[a][0] * v[0] + GB[a][1] * v[1] + GB[a][2] * v[2];
        const double pr = T[0][k] * gv[0] + T[1][k] * gv[1] + T[2][k] * gv[2];
#pragma unroll
        for (int a = 0; a < 3; ++a) v[a] -= pr * T[a][k];
      }
    double gv[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) gv[a] = GB[a][0] * v[0] + GB[a][1] * v[1] + GB[a][2] * v[2];
    const double nrm2 = v[0] * gv[0] + v[1] * gv[1] + v[2] * gv[2];
    acc[i] = n0 > 0.0 && nrm2 > drop * drop * n0;
    const double sc = acc[i] ? rsqrt(nrm2) : 0.0;
#pragma unroll
    for (int a = 0; a < 3; ++a) T[a][i] = v[a] * sc;
  }
  const int m = (int)acc[0] + (int)acc[1] + (int)acc[2];
  if (m == 0) {
    ls->status = DD_ENOTSPD;
    ls->c[0] = 1.0;
    ls->c[1] = ls->c[2] = 0.0;
    return;
  }
  double H[3][3];
#pragma unroll
  for (int p = 0; p < 3; ++p)
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      double h = 0.0;
#pragma unroll
      for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) h += T[a][p] * GA[a][b] * T[b][q];
      H[p][q] = h;
    }
  double big = 1.0;
#pragma unroll
  for (int p = 0; p < 3; ++p) {
#pragma unroll
    for (int q = p + 1; q < 3; ++q) H[p][q] = H[q][p] = 0.5 * (H[p][q] + H[q][p]);
    if (acc[p]) big += 4.0 * fabs(H[p][p]);
  }
#pragma unroll
  for (int p = 0; p < 3; ++p)
    if (!acc[p]) {   // decoupled and above every accepted Ritz value
#pragma unroll
      for (int q = 0; q < 3; ++q) H[p][q] = H[q][p] = 0.0;
      H[p][p] = big;
    }
  double theta, y[3];
  jacobi_lowest(H, &theta, y);
  double c[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) c[a] = T[a][0] * y[0] + T[a][1] * y[1] + T[a][2] * y[2];
  const double sg = ls->sums[0] * c[0] + ls->sums[1] * c[1] + ls->sums[2] * c[2];
  if (sg < 0.0)
#pragma unroll
    for (int a = 0; a < 3; ++a) c[a] = -c[a];
#pragma unroll
  for (int a = 0; a < 3; ++a) ls->c[a] = c[a];
  ls->theta = theta;
  ls->m = m;
  if (!isfinite(theta)) ls->status = DD_ENAN;
}

}  // namespace dd
