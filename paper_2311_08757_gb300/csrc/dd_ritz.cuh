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

// Lowest eigenpair of the symmetric m x m matrix H (m <= 3, row-major 3 x 3 storage) by
// cyclic Jacobi rotations (symmetric Schur decompositions of 2 x 2 blocks).
__device__ inline void jacobi_lowest(double H[3][3], int m, double* theta, double y[3]) {
  double V[3][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}};
  for (int sweep = 0; sweep < 50; ++sweep) {
    // converged once the off-diagonal mass is below the rounding of the diagonal (a rotation
    // leaves a residue of that size, so exact zeros would take all 50 sweeps of FP64
    // divisions and square roots on one thread)
    double off = 0.0, dia = 0.0;
    for (int p = 0; p < m; ++p) {
      dia += H[p][p] * H[p][p];
      for (int q = p + 1; q < m; ++q) off += H[p][q] * H[p][q];
    }
    if (off <= 1e-34 * dia) break;
    for (int p = 0; p < m; ++p)
      for (int q = p + 1; q < m; ++q) {
        const double hpq = H[p][q];
        if (hpq == 0.0) continue;
        const double dq = H[q][q] - H[p][p];
        // rotation angle: t = tan(phi) with tau = cot(2 phi).  It is formed in FP32 (GB300's
        // FP64 divide and square root are long dependent chains on one thread); normalising
        // (cs, sn) in FP64 keeps the rotation orthogonal to FP64 rounding, and an angle good
        // to FP32 still cuts H[p][q] by about 1e-7, so the sweeps above end as before
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
        for (int k = 0; k < m; ++k) {   // H <- H J
          const double hp = H[k][p], hq = H[k][q];
          H[k][p] = cs * hp - sn * hq;
          H[k][q] = sn * hp + cs * hq;
        }
        for (int k = 0; k < m; ++k) {   // H <- J^T H
          const double hp = H[p][k], hq = H[q][k];
          H[p][k] = cs * hp - sn * hq;
          H[q][k] = sn * hp + cs * hq;
        }
        for (int k = 0; k < m; ++k) {   // V <- V J
          const double vp = V[k][p], vq = V[k][q];
          V[k][p] = cs * vp - sn * vq;
          V[k][q] = sn * vp + cs * vq;
        }
      }
  }
  int lo = 0;
  for (int k = 1; k < m; ++k)
    if (H[k][k] < H[lo][lo]) lo = k;
  *theta = H[lo][lo];
  for (int k = 0; k < 3; ++k) y[k] = (k < m) ? V[k][lo] : 0.0;
}

// Orthogonalised Rayleigh-Ritz on span{x_k, w_k, x_{k-1}} from the Gram matrices (Algorithm 1):
// Gram-Schmidt in the M inner product on coefficient vectors (order x_k, w_k, x_{k-1}, two
// passes; a direction whose M-norm falls to drop times its norm before is dropped), lowest
// eigenpair of the projected matrix, coefficients signed so that the sum of the Ritz vector
// is positive.
__device__ inline void rayleigh_ritz3(LopState* ls, double drop) {
  double GA[3][3], GB[3][3];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      GA[i][j] = ls->GA[sym3(i, j)];
      GB[i][j] = ls->GB[sym3(i, j)];
    }
  double T[3][3];   // columns: accepted coefficient vectors
  int m = 0;
  for (int i = 0; i < 3; ++i) {
    double v[3] = {0.0, 0.0, 0.0};
    v[i] = 1.0;
    const double n0 = GB[i][i];
    for (int pass = 0; pass < 2; ++pass)
      for (int k = 0; k < m; ++k) {
        double gv[3];
        for (int a = 0; a < 3; ++a) gv[a] = GB[a][0] * v[0] + GB[a][1] * v[1] + GB[a][2] * v[2];
        const double pr = T[0][k] * gv[0] + T[1][k] * gv[1] + T[2][k] * gv[2];
        for (int a = 0; a < 3; ++a) v[a] -= pr * T[a][k];
      }
    double gv[3];
    for (int a = 0; a < 3; ++a) gv[a] = GB[a][0] * v[0] + GB[a][1] * v[1] + GB[a][2] * v[2];
    const double nrm2 = v[0] * gv[0] + v[1] * gv[1] + v[2] * gv[2];
    if (n0 > 0.0 && nrm2 > drop * drop * n0) {
      const double s = rsqrt(nrm2);
      for (int a = 0; a < 3; ++a) T[a][m] = v[a] * s;
      ++m;
    }
  }
  if (m == 0) {
    ls->status = DD_ENOTSPD;
    ls->c[0] = 1.0;
    ls->c[1] = ls->c[2] = 0.0;
    return;
  }
  double H[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
  for (int p = 0; p < m; ++p)
    for (int q = 0; q < m; ++q) {
      double acc = 0.0;
      for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) acc += T[a][p] * GA[a][b] * T[b][q];
      H[p][q] = acc;
    }
  for (int p = 0; p < m; ++p)
    for (int q = p + 1; q < m; ++q) H[p][q] = H[q][p] = 0.5 * (H[p][q] + H[q][p]);
  double theta, y[3];
  jacobi_lowest(H, m, &theta, y);
  double c[3];
  for (int a = 0; a < 3; ++a) {
    c[a] = 0.0;
    for (int k = 0; k < m; ++k) c[a] += T[a][k] * y[k];
  }
  const double sg = ls->sums[0] * c[0] + ls->sums[1] * c[1] + ls->sums[2] * c[2];
  if (sg < 0.0)
    for (int a = 0; a < 3; ++a) c[a] = -c[a];
  for (int a = 0; a < 3; ++a) ls->c[a] = c[a];
  ls->theta = theta;
  ls->m = m;
  if (!isfinite(theta)) ls->status = DD_ENAN;
}


}  // namespace dd
