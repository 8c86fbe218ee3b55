// SI-LOPCG outer step (Algorithm 1): Gram matrices of the search space S = [x_k, w_k, x_{k-1}]
// under A_sigma and M, the orthogonalised Rayleigh-Ritz step on them, and the update
// x_{k+1} = S c.  All three vectors, their A_sigma- and M-images are read in one pass; the
// 3 x 3 Rayleigh-Ritz problem is solved by the last block of that pass, so the coefficients
// never leave the device.
#include "dd_ritz.cuh"

namespace dd {

// Gram matrices (upper triangles) of S = [x, w, xp] under A_sigma and M, and the sums of the
// three vectors; then the Rayleigh-Ritz step in the last block.
__device__ __forceinline__ void lop_gram_body(VBlk vb, long long n, const double* __restrict__ x,
                                                       const double* __restrict__ w, const double* __restrict__ xp,
                                                       const double* __restrict__ Ax, const double* __restrict__ Aw,
                                                       const double* __restrict__ Axp, const double* __restrict__ Mx,
                                                       const double* __restrict__ Mw, const double* __restrict__ Mxp,
                                                       LopState* ls, double* partials, unsigned* counter,
                                                       double drop) {
  double acc[15];
#pragma unroll
  for (int k = 0; k < 15; ++k) acc[k] = 0.0;
  for (long long t = (long long)vb.b * blockDim.x + threadIdx.x; t < n;
       t += (long long)vb.nb * blockDim.x) {
    const double s0 = x[t], s1 = w[t], s2 = xp[t];
    const double a0 = Ax[t], a1 = Aw[t], a2 = Axp[t];
    const double m0 = Mx[t], m1 = Mw[t], m2 = Mxp[t];
    acc[0] = fma(s0, a0, acc[0]);
    acc[1] = fma(s0, a1, acc[1]);
    acc[2] = fma(s0, a2, acc[2]);
    acc[3] = fma(s1, a1, acc[3]);
    acc[4] = fma(s1, a2, acc[4]);
    acc[5] = fma(s2, a2, acc[5]);
    acc[6] = fma(s0, m0, acc[6]);
    acc[7] = fma(s0, m1, acc[7]);
    acc[8] = fma(s0, m2, acc[8]);
    acc[9] = fma(s1, m1, acc[9]);
    acc[10] = fma(s1, m2, acc[10]);
    acc[11] = fma(s2, m2, acc[11]);
    acc[12] += s0;
    acc[13] += s1;
    acc[14] += s2;
  }
  double tot[15];
  if (grid_sum_last<15>(acc, partials, counter, tot, vb) && threadIdx.x == 0) {
    for (int k = 0; k < 6; ++k) {
      ls->GA[k] = tot[k];
      ls->GB[k] = tot[6 + k];
    }
    for (int k = 0; k < 3; ++k) ls->sums[k] = tot[12 + k];
    ls->status = 0;
    bool finite = true;
    for (int k = 0; k < 15; ++k) finite = finite && isfinite(tot[k]);
    if (!finite) {
      ls->status = DD_ENAN;
      ls->c[0] = 1.0;
      ls->c[1] = ls->c[2] = 0.0;
    } else {
      rayleigh_ritz3(ls, drop);
    }
  }
}

__global__ void __launch_bounds__(kThreads) k_lop_gram(long long n, const double* __restrict__ x,
                                                       const double* __restrict__ w, const double* __restrict__ xp,
                                                       const double* __restrict__ Ax, const double* __restrict__ Aw,
                                                       const double* __restrict__ Axp, const double* __restrict__ Mx,
                                                       const double* __restrict__ Mw, const double* __restrict__ Mxp,
                                                       LopState* ls, double* partials, unsigned* counter,
                                                       double drop) {
  lop_gram_body(vblk_self(), n, x, w, xp, Ax, Aw, Axp, Mx, Mw, Mxp, ls, partials, counter, drop);
}

// out = c0 x + c1 w + c2 xp (out distinct from the inputs)
__global__ void __launch_bounds__(kThreads) k_lop_update(long long n, const double* __restrict__ x,
                                                         const double* __restrict__ w,
                                                         const double* __restrict__ xp, double* __restrict__ out,
                                                         const LopState* __restrict__ ls) {
  const double c0 = ls->c[0], c1 = ls->c[1], c2 = ls->c[2];
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n;
       t += (long long)gridDim.x * blockDim.x)
    out[t] = fma(c2, xp[t], fma(c1, w[t], c0 * x[t]));
}

// x_{k+1} = S c together with its images A_sigma x_{k+1} = (A_sigma S) c and M x_{k+1} = (M S) c
// (linear combinations instead of two more stencil passes), the outer residual
// r_o = A_sigma x - theta M x and the norms of the stop test.  c is M-normalised by the
// Rayleigh-Ritz step, so x^T M x = 1 up to rounding (its value is returned as a check).
__device__ __forceinline__ void lop_update3_body(VBlk vb, long long n, const double* __restrict__ s0,
                                                          const double* __restrict__ s1, const double* __restrict__ s2,
                                                          const double* __restrict__ a0, const double* __restrict__ a1,
                                                          const double* __restrict__ a2, const double* __restrict__ m0,
                                                          const double* __restrict__ m1, const double* __restrict__ m2,
                                                          double* __restrict__ x, double* __restrict__ ax,
                                                          double* __restrict__ mx, double* __restrict__ ro, LopState* ls,
                                                          double* partials, unsigned* counter) {
  const double c0 = ls->c[0], c1 = ls->c[1], c2 = ls->c[2], th = ls->theta;
  double acc[3] = {0.0, 0.0, 0.0};
  for (long long t = (long long)vb.b * blockDim.x + threadIdx.x; t < n;
       t += (long long)vb.nb * blockDim.x) {
    const double xv = fma(c2, s2[t], fma(c1, s1[t], c0 * s0[t]));
    const double av = fma(c2, a2[t], fma(c1, a1[t], c0 * a0[t]));
    const double mv = fma(c2, m2[t], fma(c1, m1[t], c0 * m0[t]));
    const double e = fma(-th, mv, av);
    x[t] = xv;
    ax[t] = av;
    mx[t] = mv;
    ro[t] = e;
    acc[0] = fma(e, e, acc[0]);
    acc[1] = fma(mv, mv, acc[1]);
    acc[2] = fma(xv, mv, acc[2]);
  }
  double tot[3];
  if (grid_sum_last<3>(acc, partials, counter, tot, vb) && threadIdx.x == 0) {
    ls->rr = tot[0];
    ls->mm = tot[1];
    ls->xmx = tot[2];
  }
}

__global__ void __launch_bounds__(kThreads) k_lop_update3(long long n, const double* __restrict__ s0,
                                                          const double* __restrict__ s1, const double* __restrict__ s2,
                                                          const double* __restrict__ a0, const double* __restrict__ a1,
                                                          const double* __restrict__ a2, const double* __restrict__ m0,
                                                          const double* __restrict__ m1, const double* __restrict__ m2,
                                                          double* __restrict__ x, double* __restrict__ ax,
                                                          double* __restrict__ mx, double* __restrict__ ro, LopState* ls,
                                                          double* partials, unsigned* counter) {
  lop_update3_body(vblk_self(), n, s0, s1, s2, a0, a1, a2, m0, m1, m2, x, ax, mx, ro, ls, partials, counter);
}

// in-place scaling x *= s, Mx *= s with s = os->scale (set by the normalisation dots)
__device__ __forceinline__ void lop_scale_body(VBlk vb, long long n, double* x, double* Mx, const OuterState* os) {
  const double s = os->scale;
  for (long long t = (long long)vb.b * blockDim.x + threadIdx.x; t < n;
       t += (long long)vb.nb * blockDim.x) {
    x[t] *= s;
    Mx[t] *= s;
  }
}

__global__ void __launch_bounds__(kThreads) k_lop_scale(long long n, double* x, double* Mx, const OuterState* os) {
  lop_scale_body(vblk_self(), n, x, Mx, os);
}

__global__ void k_set_entry(double* v, long long idx, double val) {
  if (threadIdx.x == 0 && blockIdx.x == 0) v[idx] = val;
}

// ---- batched forms (see k_vec.cu): the role of every vector is the same for all problems ----
__device__ __forceinline__ double* lvec(const BInst& I, int role) {
  if (role >= BV_LOP) return I.lop[role - BV_LOP];
  if (role == BV_Z) return I.z;
  if (role == BV_X) return I.x;
  return I.r;
}

struct Roles3 {
  int s[3], a[3], m[3];
};

__global__ void __launch_bounds__(kThreads) kb_lop_gram(const BInst* __restrict__ B, const int2* __restrict__ vmap,
                                                        Roles3 R, double drop) {
  const int2 m = vmap[blockIdx.x];
  const BInst& I = B[m.x];
  if (!I.active) return;
  lop_gram_body(VBlk{m.y, I.nb_vec}, I.g.plen, lvec(I, R.s[0]), lvec(I, R.s[1]), lvec(I, R.s[2]), lvec(I, R.a[0]),
                lvec(I, R.a[1]), lvec(I, R.a[2]), lvec(I, R.m[0]), lvec(I, R.m[1]), lvec(I, R.m[2]), I.lst,
                I.lop_red, I.cnt + CNT_LOP, drop);
}

__global__ void __launch_bounds__(kThreads, 4) kb_lop_update3(const BInst* __restrict__ B, const int2* __restrict__ vmap,
                                                           Roles3 R, int x_role, int ax_role, int mx_role,
                                                           int ro_role) {
  const int2 m = vmap[blockIdx.x];
  const BInst& I = B[m.x];
  if (!I.active) return;
  lop_update3_body(VBlk{m.y, I.nb_vec}, I.g.plen, lvec(I, R.s[0]), lvec(I, R.s[1]), lvec(I, R.s[2]),
                   lvec(I, R.a[0]), lvec(I, R.a[1]), lvec(I, R.a[2]), lvec(I, R.m[0]), lvec(I, R.m[1]),
                   lvec(I, R.m[2]), lvec(I, x_role), lvec(I, ax_role), lvec(I, mx_role), lvec(I, ro_role), I.lst,
                   I.lop_red, I.cnt + CNT_LOP);
}

__global__ void __launch_bounds__(kThreads) kb_lop_scale(const BInst* __restrict__ B, const int2* __restrict__ vmap,
                                                         int x_role, int mx_role) {
  const int2 m = vmap[blockIdx.x];
  const BInst& I = B[m.x];
  if (!I.active) return;
  lop_scale_body(VBlk{m.y, I.nb_vec}, I.g.plen, lvec(I, x_role), lvec(I, mx_role), I.ost);
}

__global__ void kb_lop_reset(const BInst* __restrict__ B, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n || !B[i].active) return;
  memset(B[i].lst, 0, sizeof(LopState));
  memset(B[i].ost, 0, sizeof(OuterState));
}

void launch_b_lop_gram(const BInst* B, const int2* vmap, int nvb, const int* S, const int* AS, const int* MS,
                       double drop, cudaStream_t s) {
  Roles3 R;
  for (int k = 0; k < 3; ++k) {
    R.s[k] = S[k];
    R.a[k] = AS[k];
    R.m[k] = MS[k];
  }
  (kb_lop_gram<<<nvb, kThreads, 0, s>>>(B, vmap, R, drop), dd::note_launch());
  DD_CUDA(cudaGetLastError());
}

void launch_b_lop_update3(const BInst* B, const int2* vmap, int nvb, const int* S, const int* AS, const int* MS,
                          int x_role, int ax_role, int mx_role, int ro_role, cudaStream_t s) {
  Roles3 R;
  for (int k = 0; k < 3; ++k) {
    R.s[k] = S[k];
    R.a[k] = AS[k];
    R.m[k] = MS[k];
  }
  (kb_lop_update3<<<nvb, kThreads, 0, s>>>(B, vmap, R, x_role, ax_role, mx_role, ro_role), dd::note_launch());
  DD_CUDA(cudaGetLastError());
}

// x /= ||x||_M (sign: sum x > 0) and Mx likewise: the plain lop_normalize (outer dots, scale)
void launch_b_lop_normalize(const BInst* B, const int2* vmap, int nvb, int x_role, int mx_role, cudaStream_t s) {
  launch_b_outer_dots_roles(B, vmap, nvb, x_role, mx_role, s);
  (kb_lop_scale<<<nvb, kThreads, 0, s>>>(B, vmap, x_role, mx_role), dd::note_launch());
  DD_CUDA(cudaGetLastError());
}

void launch_b_lop_reset(const BInst* B, int n, cudaStream_t s) {
  (kb_lop_reset<<<(n + 127) / 128, 128, 0, s>>>(B, n), dd::note_launch());
  DD_CUDA(cudaGetLastError());
}

void launch_lop_gram(dd_ctx* c, const double* const S[3], const double* const AS[3], const double* const MS[3],
                     double drop, cudaStream_t s) {
  const long long n = c->g.plen;
  const int nb = grid_blocks(n, kThreads);
  (k_lop_gram<<<nb, kThreads, 0, s>>>(n, S[0], S[1], S[2], AS[0], AS[1], AS[2], MS[0], MS[1], MS[2], c->lst,
                                       c->lop_red, c->cnt + CNT_LOP, drop),
   dd::note_launch());
  DD_CUDA(cudaGetLastError());
}

void launch_lop_update(dd_ctx* c, const double* x, const double* w, const double* xp, double* out,
                       cudaStream_t s) {
  const long long n = c->g.plen;
  (k_lop_update<<<grid_blocks(n, kThreads), kThreads, 0, s>>>(n, x, w, xp, out, c->lst), dd::note_launch());
  DD_CUDA(cudaGetLastError());
}

void launch_lop_update3(dd_ctx* c, const double* const S[3], const double* const AS[3], const double* const MS[3],
                        double* x, double* Ax, double* Mx, double* ro, cudaStream_t s) {
  const long long n = c->g.plen;
  (k_lop_update3<<<grid_blocks(n, kThreads), kThreads, 0, s>>>(n, S[0], S[1], S[2], AS[0], AS[1], AS[2], MS[0], MS[1],
                                                                MS[2], x, Ax, Mx, ro, c->lst, c->lop_red,
                                                                c->cnt + CNT_LOP),
   dd::note_launch());
  DD_CUDA(cudaGetLastError());
}

void launch_lop_normalize(dd_ctx* c, double* x, double* Mx, cudaStream_t s) {
  const long long n = c->g.plen;
  const int nb = grid_blocks(n, kThreads);
  launch_outer_dots(c, x, Mx, s);
  (k_lop_scale<<<nb, kThreads, 0, s>>>(n, x, Mx, c->ost), dd::note_launch());
  DD_CUDA(cudaGetLastError());
}

void launch_set_entry(double* v, long long idx, double val, cudaStream_t s) {
  (k_set_entry<<<1, 32, 0, s>>>(v, idx, val), dd::note_launch());
  DD_CUDA(cudaGetLastError());
}

}  // namespace dd
