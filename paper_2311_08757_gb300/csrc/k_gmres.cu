// Right-preconditioned restarted GMRES (flexible form: the preconditioned directions z_j are
// kept, so a rounded preconditioner is allowed) for A_sigma x = b with the two-level Schwarz
// preconditioner, the Krylov method paired with the restricted M_RAS2^{-1} (Sec. 2.2).
// Arnoldi by classical Gram-Schmidt applied twice: one pass computes all projections
// h_i = (v_i, w) (w stays in L2 while each basis vector streams from HBM once), one pass
// subtracts them.  The Givens rotations of the Hessenberg column and the triangular solve
// run in one thread on the device; the host reads only the residual estimate.
#include "dd_common.cuh"

namespace dd {

namespace {
constexpr int kDotBlocks = 304;   // blocks per projection (2 per SM)
}

// partial[i * nblk + block] = sum over this block's range of V_i[t] w[t], i < nv
__global__ void __launch_bounds__(kThreads) k_multidot(long long n, int nv, const double* const* __restrict__ V,
                                                       const double* __restrict__ w, double* partial) {
  const long long per = (n + gridDim.x - 1) / gridDim.x;
  const long long t0 = blockIdx.x * per, t1 = min(n, t0 + per);
  for (int i = 0; i < nv; ++i) {
    const double* vi = V[i];
    double acc[1] = {0.0};
    for (long long t = t0 + threadIdx.x; t < t1; t += blockDim.x) acc[0] = fma(vi[t], w[t], acc[0]);
    block_sum<1>(acc);
    if (threadIdx.x == 0) partial[(size_t)i * gridDim.x + blockIdx.x] = acc[0];
  }
}

// h[i] (+)= sum over blocks of partial[i][.], in block order; one block per i
__global__ void k_multidot_finish(int nblk, const double* __restrict__ partial, double* h, int accumulate) {
  const int i = blockIdx.x;
  double acc[1] = {0.0};
  for (int b = threadIdx.x; b < nblk; b += blockDim.x) acc[0] += partial[(size_t)i * nblk + b];
  block_sum<1>(acc);
  if (threadIdx.x == 0) h[i] = accumulate ? h[i] + acc[0] : acc[0];
}

// w[t] -= sum_i coef[i] V_i[t]   (sign = -1), or x[t] += sum_i coef[i] V_i[t] (sign = +1)
__global__ void __launch_bounds__(kThreads) k_multiaxpy(long long n, int nv, const double* const* __restrict__ V,
                                                        const double* __restrict__ coef, double sign, double* w) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n;
       t += (long long)gridDim.x * blockDim.x) {
    double acc = 0.0;
    for (int i = 0; i < nv; ++i) acc = fma(__ldg(coef + i), V[i][t], acc);
    w[t] = fma(sign, acc, w[t]);
  }
}

// v = w / ||w||, the squared norm read from the device
__global__ void __launch_bounds__(kThreads) k_scale_by_norm(long long n, const double* __restrict__ w,
                                                            const double* __restrict__ nrm2, double* v) {
  const double nv = sqrt(*nrm2);
  const double s = nv > 0.0 ? 1.0 / nv : 0.0;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n;
       t += (long long)gridDim.x * blockDim.x)
    v[t] = w[t] * s;
}

// Column j of the Hessenberg matrix (h[0..j] from the projections, ||w||^2 in nrm2): apply the
// earlier rotations, form the new one, update g; res[0] = |g[j+1]| (residual estimate).
// H is column-major with leading dimension ld = restart + 1.
__global__ void k_givens(int j, int ld, const double* __restrict__ h, const double* __restrict__ nrm2, double* H,
                         double* cs, double* sn, double* g, double* res) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double* col = H + (size_t)j * ld;
  for (int i = 0; i <= j; ++i) col[i] = h[i];
  col[j + 1] = sqrt(*nrm2);
  for (int i = 0; i < j; ++i) {
    const double t = cs[i] * col[i] + sn[i] * col[i + 1];
    col[i + 1] = -sn[i] * col[i] + cs[i] * col[i + 1];
    col[i] = t;
  }
  const double a = col[j], b = col[j + 1];
  const double den = hypot(a, b);
  const double c = den > 0.0 ? a / den : 1.0, s = den > 0.0 ? b / den : 0.0;
  cs[j] = c;
  sn[j] = s;
  col[j] = den;
  col[j + 1] = 0.0;
  g[j + 1] = -s * g[j];
  g[j] = c * g[j];
  res[0] = fabs(g[j + 1]);
}

// y = R^{-1} g (R the rotated Hessenberg, m x m upper triangle), then the update coefficients
__global__ void k_backsolve(int m, int ld, const double* __restrict__ H, const double* __restrict__ g, double* y) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  for (int i = m - 1; i >= 0; --i) {
    double acc = g[i];
    for (int k = i + 1; k < m; ++k) acc -= H[(size_t)k * ld + i] * y[k];
    y[i] = acc / H[(size_t)i * ld + i];
  }
}

// g = (beta, 0, ...) with beta = sqrt(nrm2)
__global__ void k_gmres_start(const double* __restrict__ nrm2, double* g, int len) {
  for (int i = threadIdx.x; i < len; i += blockDim.x) g[i] = (i == 0) ? sqrt(*nrm2) : 0.0;
}

__global__ void k_add_inplace(int n, double* a, const double* __restrict__ b) {
  for (int i = threadIdx.x; i < n; i += blockDim.x) a[i] += b[i];
}

void launch_add_inplace(dd_ctx* c, int n, double* a, const double* b, cudaStream_t s) {
  (void)c;
  (k_add_inplace<<<1, 64, 0, s>>>(n, a, b), dd::note_launch());
  DD_CUDA(cudaGetLastError());
}

void launch_multidot(dd_ctx* c, int nv, const double* const* V, const double* w, double* h, int accumulate,
                     cudaStream_t s) {
  const long long n = c->g.plen;
  (k_multidot<<<kDotBlocks, kThreads, 0, s>>>(n, nv, V, w, c->gm_part), dd::note_launch());
  (k_multidot_finish<<<nv, 256, 0, s>>>(kDotBlocks, c->gm_part, h, accumulate), dd::note_launch());
  DD_CUDA(cudaGetLastError());
}

void launch_multiaxpy(dd_ctx* c, int nv, const double* const* V, const double* coef, double sign, double* w,
                      cudaStream_t s) {
  const long long n = c->g.plen;
  (k_multiaxpy<<<grid_blocks(n, kThreads), kThreads, 0, s>>>(n, nv, V, coef, sign, w), dd::note_launch());
  DD_CUDA(cudaGetLastError());
}

void launch_scale_by_norm(dd_ctx* c, const double* w, const double* nrm2, double* v, cudaStream_t s) {
  const long long n = c->g.plen;
  (k_scale_by_norm<<<grid_blocks(n, kThreads), kThreads, 0, s>>>(n, w, nrm2, v), dd::note_launch());
  DD_CUDA(cudaGetLastError());
}

void launch_givens(dd_ctx* c, int j, cudaStream_t s) {
  const int ld = c->gm_restart + 1;
  // h[0..j] at gm_h, ||w||^2 at gm_h + 2 ld (the second pass's projections at gm_h + ld)
  (k_givens<<<1, 32, 0, s>>>(j, ld, c->gm_h, c->gm_h + 2 * ld, c->gm_H, c->gm_cs, c->gm_sn, c->gm_g, c->gm_res),
   dd::note_launch());
  DD_CUDA(cudaGetLastError());
}

void launch_backsolve(dd_ctx* c, int m, cudaStream_t s) {
  const int ld = c->gm_restart + 1;
  (k_backsolve<<<1, 32, 0, s>>>(m, ld, c->gm_H, c->gm_g, c->gm_y), dd::note_launch());
  DD_CUDA(cudaGetLastError());
}

void launch_gmres_start(dd_ctx* c, const double* nrm2, cudaStream_t s) {
  (k_gmres_start<<<1, 64, 0, s>>>(nrm2, c->gm_g, c->gm_restart + 1), dd::note_launch());
  DD_CUDA(cudaGetLastError());
}

}  // namespace dd
