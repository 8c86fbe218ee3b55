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

// The same rotation in FP32 (for the first, FP32 pass of lowest_eigenpair3)
template <int p, int q>
__device__ __forceinline__ void jacobi_rotate_f(float (&F)[3][3], float (&V)[3][3]) {
  const float fpq = F[p][q];
  if (fpq == 0.0f) return;
  const float tau = (F[q][q] - F[p][p]) / (2.0f * fpq);
  const float t = copysignf(1.0f, tau) / (fabsf(tau) + sqrtf(fmaf(tau, tau, 1.0f)));
  const float cs = rsqrtf(fmaf(t, t, 1.0f)), sn = t * cs;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const float hp = F[k][p], hq = F[k][q];
    F[k][p] = cs * hp - sn * hq;
    F[k][q] = sn * hp + cs * hq;
  }
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const float hp = F[p][k], hq = F[q][k];
    F[p][k] = cs * hp - sn * hq;
    F[q][k] = sn * hp + cs * hq;
  }
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const float vp = V[k][p], vq = V[k][q];
    V[k][p] = cs * vp - sn * vq;
    V[k][q] = sn * vp + cs * vq;
  }
}

// Lowest eigenpair of the symmetric 3 x 3 matrix H, at FP64 accuracy with few FP64
// instructions (a lone thread issues one FP64 warp instruction per ~64 cycles on GB300, while
// FP32 instructions are cheap): cyclic Jacobi sweeps in FP32 on H scaled to unit size give
// the eigenvector to about 1e-7; one Rayleigh-quotient step in FP64 refines it, z = adj(H -
// theta I) y with theta the Rayleigh quotient of y (the adjugate of the nearly singular
// shifted matrix maps every vector onto the eigenvector: inverse iteration without a solve);
// a residual check accepts the result, else the FP64 Jacobi sweeps decide (a degenerate or
// nearly degenerate lowest pair).
__device__ inline void lowest_eigenpair3(double (&H)[3][3], double* theta, double (&y)[3]) {
  double s = 0.0;
#pragma unroll
  for (int p = 0; p < 3; ++p)
#pragma unroll
    for (int q = p; q < 3; ++q) s = fmax(s, fabs(H[p][q]));
  if (!(s > 0.0) || !isfinite(s)) {
    jacobi_lowest(H, theta, y);
    return;
  }
  const double is = 1.0 / s;
  float F[3][3], Vf[3][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}};
#pragma unroll
  for (int p = 0; p < 3; ++p)
#pragma unroll
    for (int q = 0; q < 3; ++q) F[p][q] = (float)(H[p][q] * is);
#pragma unroll 1
  for (int sweep = 0; sweep < 12; ++sweep) {
    const float off = F[0][1] * F[0][1] + F[0][2] * F[0][2] + F[1][2] * F[1][2];
    if (off <= 1e-14f) break;
    jacobi_rotate_f<0, 1>(F, Vf);
    jacobi_rotate_f<0, 2>(F, Vf);
    jacobi_rotate_f<1, 2>(F, Vf);
  }
  const int lo = (F[0][0] <= F[1][1]) ? ((F[0][0] <= F[2][2]) ? 0 : 2) : ((F[1][1] <= F[2][2]) ? 1 : 2);
  double v[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) v[k] = (double)((lo == 0) ? Vf[k][0] : ((lo == 1) ? Vf[k][1] : Vf[k][2]));
  // Rayleigh quotient of v, then z = adj(H - th I) v
  double hv[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) hv[a] = H[a][0] * v[0] + H[a][1] * v[1] + H[a][2] * v[2];
  const double th = (v[0] * hv[0] + v[1] * hv[1] + v[2] * hv[2]) / (v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
  const double a00 = H[0][0] - th, a11 = H[1][1] - th, a22 = H[2][2] - th;
  const double a01 = H[0][1], a02 = H[0][2], a12 = H[1][2];
  const double c00 = a11 * a22 - a12 * a12, c11 = a00 * a22 - a02 * a02, c22 = a00 * a11 - a01 * a01;
  const double c01 = a02 * a12 - a01 * a22, c02 = a01 * a12 - a02 * a11, c12 = a01 * a02 - a00 * a12;
  double z[3] = {c00 * v[0] + c01 * v[1] + c02 * v[2], c01 * v[0] + c11 * v[1] + c12 * v[2],
                 c02 * v[0] + c12 * v[1] + c22 * v[2]};
  const double zz = z[0] * z[0] + z[1] * z[1] + z[2] * z[2];
  bool good = zz > 0.0 && isfinite(zz);
  if (good) {
    const double rz = rsqrt(zz);
#pragma unroll
    for (int a = 0; a < 3; ++a) z[a] *= rz;
    double hz[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) hz[a] = H[a][0] * z[0] + H[a][1] * z[1] + H[a][2] * z[2];
    const double tz = z[0] * hz[0] + z[1] * hz[1] + z[2] * hz[2];
    double res = 0.0;
#pragma unroll
    for (int a = 0; a < 3; ++a) res = fma(hz[a] - tz * z[a], hz[a] - tz * z[a], res);
    // accept at the rounding level of H (the Jacobi route reaches the same)
    good = res <= 1e-26 * s * s && tz <= th + 1e-12 * s;
    if (good) {
      *theta = tz;
#pragma unroll
      for (int a = 0; a < 3; ++a) y[a] = z[a];
      return;
    }
  }
  jacobi_lowest(H, theta, y);
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
  // H = T^T (GA T): upper triangle only (H is symmetric)
  double G2[3][3];
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int q = 0; q < 3; ++q) G2[a][q] = GA[a][0] * T[0][q] + GA[a][1] * T[1][q] + GA[a][2] * T[2][q];
  double H[3][3];
#pragma unroll
  for (int p = 0; p < 3; ++p)
#pragma unroll
    for (int q = p; q < 3; ++q) H[p][q] = H[q][p] = T[0][p] * G2[0][q] + T[1][p] * G2[1][q] + T[2][p] * G2[2][q];
  double big = 1.0;
#pragma unroll
  for (int p = 0; p < 3; ++p)
    if (acc[p]) big += 4.0 * fabs(H[p][p]);
#pragma unroll
  for (int p = 0; p < 3; ++p)
    if (!acc[p]) {   // decoupled and above every accepted Ritz value
#pragma unroll
      for (int q = 0; q < 3; ++q) H[p][q] = H[q][p] = 0.0;
      H[p][p] = big;
    }
  double theta, y[3];
  lowest_eigenpair3(H, &theta, y);
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
