// PerFact coarse space (Definition 2.1): R_0^T = blockdiag(D_i R_i psi), one column per
// subdomain; coarse matrix A_{sigma,0} = R_0 A_sigma R_0^T and its solve (Sec. 3.1).
//
// The weights D_i R_i psi of all subdomains of one type are the same table (the cells are
// translated copies, psi and the partition of unity are periodic), stored per type.
// A_0 couples only neighbouring subdomains (supports of D_i R_i psi overlap only for
// |i - j| <= 1 per axis since 2 delta < n), so it is assembled with 3^p coloured
// operator applications: v_c = sum of the columns of colour c, w_c = A_sigma v_c, and
// A_0[i][j] = (D_i R_i psi)^T w_{c(j)} for the unique neighbour j of i of colour c.
//   p = 1: A_0 is tridiagonal, solved by cyclic reduction in one CTA (coefficients
//          precomputed once, so each solve is 2 log2 N synchronised sweeps).
//   p = 2: A_0 is block tridiagonal (bandwidth L + 1); its dense inverse is formed once
//          from a banded Cholesky factor and applied as an FP64 matrix-vector product.
#include <atomic>

#include "dd_async.cuh"
#include "dd_band.cuh"

namespace dd {

// Distance of a node coordinate to the artificial faces of subdomain i along one axis
// (Sec. 4.1.2: d_i = dist(z, dOmega_i minus dOmega) inside Omega_i); +inf if no face.
__device__ inline double axis_face_dist(const Geo& g, int i, int a) {
  const double x = a * g.h;
  const double lo = i - g.delta * g.h, hi = i + 1 + g.delta * g.h;
  double d = 1e300;
  if (lo > 1e-12) d = fmin(d, x - lo);
  if (hi < g.L - 1e-12) d = fmin(d, hi - x);
  return d;
}

// partition-of-unity weight of subdomain (i1, i2) at node (a1, a2)
__device__ double pu_weight(const Geo& g, int pu, int i1, int i2, int a1, int a2) {
  int o1[2], l1[2], o2[2] = {0, 0}, l2[2] = {0, 0};
  const int n1 = axis_owners(g, a1, o1, l1);
  const int n2 = (g.p == 2) ? axis_owners(g, a2, o2, l2) : 1;
  if (pu == DD_PU_EQUAL) return 1.0 / (double)(n1 * n2);
  if (g.nsub == 1) return 1.0;
  double mine = 0.0, tot = 0.0;
  for (int i = 0; i < n1; ++i)
    for (int k = 0; k < n2; ++k) {
      double d = axis_face_dist(g, o1[i], a1);
      if (g.p == 2) d = fmin(d, axis_face_dist(g, o2[k], a2));
      tot += d;
      if (o1[i] == i1 && (g.p == 1 || o2[k] == i2)) mine = d;
    }
  return mine / tot;
}

__global__ void k_coarse_weights(Geo g, int pu, const Sub* __restrict__ rep, int ntypes, int kpad,
                                 const double* __restrict__ psi, double* wT, double* puT,
                                 float* wT32, float* puT32) {
  const long long total = (long long)ntypes * kpad;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const int ty = (int)(t / kpad), kp = (int)(t % kpad);   // column-padded local index
    const Sub s = rep[ty];
    double v = 0.0, d = 0.0;
    const int sj = kp & (g.Ypad - 1), cc = kp >> g.ylog;
    if (sj < g.nyi && cc < s.w1 * s.w2) {
      const int c1 = cc / s.w2, c2 = cc % s.w2;
      const int a1 = s.lo1 + c1, a2 = s.lo2 + c2;
      // subdomain index of the representative along each axis: from its first column
      const int i1 = (s.lo1 + g.delta - 1) / g.n, i2 = (g.p == 2) ? (s.lo2 + g.delta - 1) / g.n : 0;
      int pc;
      if (g.p == 1) pc = (a1 % g.n) * g.nyi + sj;
      else pc = ((a1 % g.n) * g.n + (a2 % g.n)) * g.nyi + sj;
      d = pu_weight(g, pu, i1, i2, a1, a2);
      v = d * psi[pc];
    }
    wT[t] = v;     // D_i R_i psi: the coarse basis function of the type
    puT[t] = d;    // D_i: the partition-of-unity weights (restricted local prolongation)
    wT32[t] = __double2float_rn(v);
    puT32[t] = __double2float_rn(d);
  }
}

static Sub* upload_reps(dd_ctx* c) {
  std::vector<Sub> rep(c->ntypes);
  for (int t = 0; t < c->ntypes; ++t)
    for (const Sub& s : c->subs_h)
      if (s.type == t) { rep[t] = s; break; }
  Sub* d = nullptr;
  DD_CUDA(cudaMallocAsync(&d, sizeof(Sub) * c->ntypes, c->stream));
  DD_CUDA(cudaMemcpyAsync(d, rep.data(), sizeof(Sub) * c->ntypes, cudaMemcpyHostToDevice, c->stream));
  return d;
}

void launch_coarse_weights(dd_ctx* c) {
  Sub* rep = upload_reps(c);
  const long long total = (long long)c->ntypes * c->kpad;
  (k_coarse_weights<<<grid_blocks(total, 128), 128, 0, c->stream>>>(c->g, c->grid.pu_kind, rep, c->ntypes,
                                                                   c->kpad, c->psi_cell, c->wT, c->puT, c->wT32,
                                                                   c->puT32), dd::note_launch());
  DD_CUDA(cudaGetLastError());
  DD_CUDA(cudaFreeAsync(rep, c->stream));
}

// local index k of subdomain s -> padded global index
__device__ __forceinline__ long long sub_global(const Geo& g, const Sub& sb, int k) {
  const int sj = k % g.nyi, cc = k / g.nyi;
  const int c1 = cc / sb.w2, c2 = cc % sb.w2;
  if (g.p == 1) return (long long)(sb.lo1 + c1) * g.Ypad + sj;
  return ((long long)(sb.lo1 + c1) * g.ncx + (sb.lo2 + c2)) * g.Ypad + sj;
}

// v = sum of the coarse columns of colour (c1, c2)
__global__ void k_colour_vector(Geo g, const Sub* __restrict__ subs, const double* __restrict__ wT, int kpad,
                                int col1, int col2, double* v) {
  const long long total = (long long)g.nxi * (g.p == 2 ? g.nxi : 1) * g.Ypad;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    Node nd = (g.p == 1) ? node_of<1>(g, t) : node_of<2>(g, t);
    double val = 0.0;
    if (nd.slot < g.nyi) {
      int o1[2], l1[2], o2[2] = {0, 0}, l2[2] = {0, 0};
      const int n1 = axis_owners(g, nd.a1, o1, l1);
      const int n2 = (g.p == 2) ? axis_owners(g, nd.a2, o2, l2) : 1;
      for (int i = 0; i < n1; ++i)
        for (int k = 0; k < n2; ++k) {
          if (o1[i] % 3 != col1) continue;
          if (g.p == 2 && o2[k] % 3 != col2) continue;
          const int s = (g.p == 1) ? o1[i] : o1[i] * g.L + o2[k];
          const Sub sb = subs[s];
          const int loc = ((g.p == 1) ? l1[i] : l1[i] * sb.w2 + l2[k]) * g.Ypad + nd.slot;
          val += wT[(size_t)sb.type * kpad + loc];
        }
    }
    v[nd.idx] = val;
  }
}

// A0nb[s][nb] for the neighbour of colour (col1, col2): block per subdomain
__global__ void k_coarse_entries(Geo g, const Sub* __restrict__ subs, const double* __restrict__ wT, int kpad,
                                 int col1, int col2, const double* __restrict__ w, double* A0nb) {
  const int s = blockIdx.x;
  const int s1 = (g.p == 1) ? s : s / g.L, s2 = (g.p == 1) ? 0 : s % g.L;
  // the neighbour of colour col along each axis
  int t1 = -10, t2 = 0;
  for (int d = -1; d <= 1; ++d)
    if (((s1 + d) % 3 + 3) % 3 == col1) t1 = s1 + d;
  if (g.p == 2) {
    t2 = -10;
    for (int d = -1; d <= 1; ++d)
      if (((s2 + d) % 3 + 3) % 3 == col2) t2 = s2 + d;
  }
  if (t1 < 0 || t1 >= g.L || (g.p == 2 && (t2 < 0 || t2 >= g.L))) return;
  const Sub sb = subs[s];
  double acc[1] = {0.0};
  for (int k = threadIdx.x; k < sb.nloc; k += blockDim.x)
    acc[0] = fma(wT[(size_t)sb.type * kpad + loc_pad(g, k)], w[sub_global(g, sb, k)], acc[0]);
  block_sum<1>(acc);
  if (threadIdx.x == 0) {
    const int nbk = (g.p == 1) ? (t1 - s1 + 1) : ((t1 - s1 + 1) * 3 + (t2 - s2 + 1));
    A0nb[(size_t)s * (g.p == 1 ? 3 : 9) + nbk] = acc[0];
  }
}

int coarse_assemble(dd_ctx* c, cudaStream_t s) {
  const Geo& g = c->g;
  const int nnb = (g.p == 1) ? 3 : 9;
  DD_CUDA(cudaMemsetAsync(c->A0band, 0, sizeof(double) * (size_t)g.nsub * nnb, s));
  const long long work = (long long)g.nxi * (g.p == 2 ? g.nxi : 1) * g.Ypad;
  const int ncol2 = (g.p == 2) ? 3 : 1;
  for (int c1 = 0; c1 < 3; ++c1)
    for (int c2 = 0; c2 < ncol2; ++c2) {
      (k_colour_vector<<<grid_blocks(work, kThreads), kThreads, 0, s>>>(g, c->subs, c->wT, c->kpad, c1, c2, c->w1),
       dd::note_launch());
      launch_stencil(c, c->tabS, c->w1, c->w2, s);
      (k_coarse_entries<<<g.nsub, 256, 0, s>>>(g, c->subs, c->wT, c->kpad, c1, c2, c->w2, c->A0band),
       dd::note_launch());
      DD_CUDA(cudaGetLastError());
    }
  return DD_OK;
}

// ----------------------------------------------------------------------------------------
// p = 1: cyclic reduction for the tridiagonal A_0 (symmetric positive definite, so the
// odd-even elimination needs no pivoting).  Equations j = 1..N:
// a_j x_{j-1} + b_j x_j + c_j x_{j+1} = f_j, x_0 = x_{N+1} = 0.  Level l (stride s = 2^l)
// eliminates x_{j-s}, x_{j+s} from the equations j = 2s, 4s, ... <= N with multipliers
// alpha, gamma, stored packed per level (N >> (l+1) each); the levels run up to the root
// 2^(m-1) <= N (2^m - 1 >= N).  Indices beyond N stand for identity rows (b = 1, a = c = 0,
// f = 0), the usual padding to 2^m - 1 equations, which is never stored or computed.
// Layout of c->cr (each array a multiple of two doubles, so every array starts 16-byte
// aligned): alpha[C2], gamma[C2], a[W2], binv[W2], cc[W2], then b[W2] (set-up work),
// C2 >= sum of the per-level counts, W2 >= N + 2.
// ----------------------------------------------------------------------------------------
__device__ __forceinline__ int cr_count(int N, int l) { return N >> (l + 1); }

__global__ void __launch_bounds__(1024) k_cr_setup(const double* __restrict__ A0nb, int N, int m, int C2, int W2,
                                                   double* cr, int* flag) {
  double* alpha = cr;
  double* gamma = cr + C2;
  double* a = cr + 2 * (size_t)C2;
  double* binv = a + W2;
  double* cc = binv + W2;
  double* b = cc + W2;   // work: b values
  for (int j = threadIdx.x; j < W2; j += blockDim.x) {
    double aj = 0.0, bj = 1.0, cj = 0.0;
    if (j >= 1 && j <= N) {
      bj = A0nb[(size_t)(j - 1) * 3 + 1];
      aj = (j >= 2) ? A0nb[(size_t)(j - 1) * 3 + 0] : 0.0;
      cj = (j <= N - 1) ? A0nb[(size_t)(j - 1) * 3 + 2] : 0.0;
    }
    a[j] = aj;
    b[j] = bj;
    cc[j] = cj;
  }
  __syncthreads();
  int off = 0;
  for (int l = 0; l < m - 1; ++l) {
    const int s = 1 << l;
    const int cnt = cr_count(N, l);
    for (int t = threadIdx.x; t < cnt; t += blockDim.x) {
      const int j = 2 * s * (t + 1);
      const bool in = j + s <= N;   // otherwise x_{j+s} is a padding unknown
      const double bp = in ? b[j + s] : 1.0, ap = in ? a[j + s] : 0.0, cp = in ? cc[j + s] : 0.0;
      const double al = -a[j] / b[j - s];
      const double ga = -cc[j] / bp;
      alpha[off + t] = al;
      gamma[off + t] = ga;
      b[j] = b[j] + al * cc[j - s] + ga * ap;
      a[j] = al * a[j - s];
      cc[j] = ga * cp;
    }
    off += cnt;
    __syncthreads();
  }
  for (int j = threadIdx.x; j < W2; j += blockDim.x) {
    if (!(b[j] > 0.0)) atomicOr(flag, 1);
    binv[j] = 1.0 / b[j];
  }
}

constexpr int kCrThreads = 512;
constexpr int ERR_CR_WAIT = 1 << 7;   // error-word bit: the coefficient copy did not arrive in time

// The coefficients are brought into shared memory by bulk copies (the TMA engine, one
// thread issues them) while the threads load the right-hand side; every level then waits on
// shared memory only.  When they do not fit (very long chains), they are read from global.
__device__ __forceinline__ void cr_solve_body(const double* __restrict__ cr, int N, int m, int C2, int W2,
                                              const double* __restrict__ rhs, double* __restrict__ x,
                                              float* __restrict__ xf, const PcgState* st, int staged, int* err) {
  // the converged flag is tested once the copies have landed, so that its load overlaps them
  const int done = (st != nullptr) ? st->done : 0;
  extern __shared__ __align__(16) double sm_cr[];
  __shared__ __align__(8) unsigned long long cr_bar;
  __shared__ int cr_ok;
  double* f = sm_cr;
  const size_t ncoef = 2 * (size_t)C2 + 3 * (size_t)W2;
  const double* src = cr;
  if (staged) {
    const uint32_t bar = smem_u32(&cr_bar);
    if (threadIdx.x == 0) {
      mbar_init(bar, 1);
      asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      const uint32_t total = (uint32_t)(ncoef * sizeof(double));
      mbar_expect_tx(bar, total);
      const uint32_t dst = smem_u32(sm_cr + W2);
      constexpr uint32_t kChunk = 32768;
      for (uint32_t o = 0; o < total; o += kChunk)
        bulk_g2s(dst + o, reinterpret_cast<const char*>(cr) + o, min(kChunk, total - o), bar);
    }
    src = sm_cr + W2;
  }
  for (int j = threadIdx.x; j < W2; j += blockDim.x) f[j] = (j >= 1 && j <= N) ? rhs[j - 1] : 0.0;
  if (staged) {
    if (threadIdx.x == 0) cr_ok = mbar_wait(smem_u32(&cr_bar), 0, err, ERR_CR_WAIT) ? 1 : 0;
  } else if (threadIdx.x == 0) {
    cr_ok = 1;
  }
  __syncthreads();
  if (!cr_ok || done) return;   // the error word tells the host
  const double* alpha = src;
  const double* gamma = src + C2;
  const double* a = src + 2 * (size_t)C2;
  const double* binv = a + W2;
  const double* cc = binv + W2;
  int off = 0;
  for (int l = 0; l < m - 1; ++l) {
    const int s = 1 << l;
    const int cnt = cr_count(N, l);
    for (int t = threadIdx.x; t < cnt; t += blockDim.x) {
      const int j = 2 * s * (t + 1);
      const double fp = (j + s <= N) ? f[j + s] : 0.0;
      f[j] = fma(alpha[off + t], f[j - s], fma(gamma[off + t], fp, f[j]));
    }
    off += cnt;
    __syncthreads();
  }
  const int root = 1 << (m - 1);
  if (threadIdx.x == 0) f[root] *= binv[root];
  __syncthreads();
  for (int l = m - 2; l >= 0; --l) {
    const int s = 1 << l;
    for (int j = s + 2 * s * threadIdx.x; j <= N; j += 2 * s * blockDim.x) {
      const double left = f[j - s];
      const double right = (j + s <= N) ? f[j + s] : 0.0;
      f[j] = (f[j] - a[j] * left - cc[j] * right) * binv[j];
    }
    __syncthreads();
  }
  for (int j = threadIdx.x; j < N; j += blockDim.x) {
    x[j] = f[j + 1];
    xf[j] = __double2float_rn(f[j + 1]);
  }
}

__global__ void __launch_bounds__(kCrThreads) k_cr_solve(const double* __restrict__ cr, int N, int m, int C2,
                                                         int W2, const double* __restrict__ rhs,
                                                         double* __restrict__ x, float* __restrict__ xf,
                                                         const PcgState* st, int staged, int* err) {
  cr_solve_body(cr, N, m, C2, W2, rhs, x, xf, st, staged, err);
}

// batched: one CTA per problem
__global__ void __launch_bounds__(kCrThreads) kb_cr_solve(const BInst* __restrict__ B) {
  const BInst& I = B[blockIdx.x];
  if (!I.active) return;
  cr_solve_body(I.cr, I.nsub, I.cr_m, I.cr_c2, I.cr_w2, I.c0, I.u0, I.u0f, I.st, I.cr_staged, I.err + 8);
}

// dense inverse rows from the banded factor (identity right-hand sides, K per warp)
template <typename T, int NV, int PF, int K>
__global__ void k_band_inverse_rows(int n, int b, const T* __restrict__ CB, const T* __restrict__ RB,
                                    const T* __restrict__ inv, T* out) {
  extern __shared__ __align__(16) unsigned char xs_raw[];
  T* xs_all = reinterpret_cast<T*>(xs_raw);
  const int wpb = blockDim.x >> 5, wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int col0 = (blockIdx.x * wpb + wid) * K;
  if (col0 >= n) return;
  constexpr int RING = band_ring_elems<NV, PF>();
  T* xs = xs_all + (size_t)wid * (K * n + RING);
  T* ring = xs + (size_t)K * n;
#pragma unroll
  for (int j = 0; j < K; ++j)
    for (int k = lane; k < n; k += 32) xs[(size_t)j * n + k] = (k == col0 + j) ? (T)1 : (T)0;
  band_solve_k<NV, PF, K>(xs, n, n, b, CB, RB, inv, ring);
  __syncwarp();
  for (int j = 0; j < K && col0 + j < n; ++j)
    for (int k = lane; k < n; k += 32) out[(size_t)(col0 + j) * n + k] = xs[(size_t)j * n + k];
}

template <typename T>
void launch_band_inverse_rows(int n, int b, const T* CB, const T* RB, const T* inv, T* out, cudaStream_t s) {
  DD_BAND_DISPATCH(b, {
    // one identity column per warp: the warps, not the columns per warp, hide the latency of
    // the sequential steps here (992 columns; four per warp measured 262 against 176 us)
    constexpr int KK = 1;
    const size_t per = sizeof(T) * (size_t)KK * n + band_ring_bytes(b, sizeof(T));
    const int wpb = per <= 48 * 1024 ? 2 : 1;
    const size_t smem = per * wpb;
    const int ncolgroups = (n + KK - 1) / KK;
    DD_CUDA(cudaFuncSetAttribute(k_band_inverse_rows<T, NV, PF, KK>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 220 * 1024));
    (k_band_inverse_rows<T, NV, PF, KK><<<(ncolgroups + wpb - 1) / wpb, 32 * wpb, smem, s>>>(n, b, CB, RB, inv, out),
     dd::note_launch());
  });
  DD_CUDA(cudaGetLastError());
}
template void launch_band_inverse_rows<double>(int, int, const double*, const double*, const double*, double*,
                                               cudaStream_t);
template void launch_band_inverse_rows<float>(int, int, const float*, const float*, const float*, float*,
                                              cudaStream_t);

__global__ void k_gemv_rows(int n, const double* __restrict__ A, const double* __restrict__ xin,
                            double* __restrict__ y, float* __restrict__ yf, const PcgState* st) {
  if (st != nullptr && st->done) return;
  const int wpb = blockDim.x >> 5, wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int row = blockIdx.x * wpb + wid;
  if (row >= n) return;
  const double* ar = A + (size_t)row * n;
  double acc = 0.0;
  for (int k = lane; k < n; k += 32) acc = fma(ar[k], __ldg(xin + k), acc);
  acc = warp_sum(acc);
  if (lane == 0) {
    y[row] = acc;
    if (yf != nullptr) yf[row] = __double2float_rn(acc);
  }
}

int coarse_factor(dd_ctx* c) {
  const Geo& g = c->g;
  const int N = g.nsub;
  int* flag = c->dev_err + 2;
  DD_CUDA(cudaMemsetAsync(flag, 0, sizeof(int), c->stream));
  c->coarse_dense = (g.p == 2) || c->coarse_mode == 2;
  if (!c->coarse_dense) {
    int m = 1;
    while ((1 << m) - 1 < N) ++m;
    int C = 0;
    for (int l = 0; l < m - 1; ++l) C += N >> (l + 1);
    const int C2 = (C + 1) & ~1, W2 = (N + 3) & ~1;
    c->cr_m = m;
    c->cr_c2 = C2;
    c->cr_w2 = W2;
    if (!c->cr) c->cr = (double*)dev_alloc(c, sizeof(double) * (2 * (size_t)C2 + 4 * (size_t)W2));   // kept across builds
    (k_cr_setup<<<1, 1024, 0, c->stream>>>(c->A0band, N, m, C2, W2, c->cr, flag), dd::note_launch());
    DD_CUDA(cudaGetLastError());
  } else {
    // dense A_0^{-1} (rows from the banded Cholesky factor), applied as a GEMV in the solve
    const int b = (g.p == 2) ? g.L + 1 : 1;
    const int nn = (g.p == 2) ? 9 : 3;   // couplings per coarse row
    const size_t cb = sizeof(double) * (size_t)N * (b + 1);
    if (!c->cf_CB) {   // kept across builds (same grid)
      c->cf_CB = (double*)dev_alloc(c, cb);
      c->cf_RB = (double*)dev_alloc(c, cb);
      c->cf_inv = (double*)dev_alloc(c, sizeof(double) * N);
    }
    double *CB = c->cf_CB, *RB = c->cf_RB, *inv = c->cf_inv;
    // scatter the 3- or 9-point coarse rows into lower band storage (order s = s1 L + s2)
    std::vector<double> nb((size_t)N * nn), hcb((size_t)N * (b + 1), 0.0);
    DD_CUDA(cudaMemcpyAsync(nb.data(), c->A0band, sizeof(double) * N * nn, cudaMemcpyDeviceToHost, c->stream));
    DD_CUDA(cudaStreamSynchronize(c->stream));
    for (int s = 0; s < N; ++s) {
      const int s1 = (g.p == 2) ? s / g.L : s, s2 = (g.p == 2) ? s % g.L : 0;
      for (int k = 0; k < nn; ++k) {
        const int t1 = s1 + (g.p == 2 ? k / 3 : k) - 1, t2 = (g.p == 2) ? s2 + k % 3 - 1 : 0;
        if (t1 < 0 || t1 >= ((g.p == 2) ? g.L : N) || t2 < 0 || (g.p == 2 && t2 >= g.L)) continue;
        const int t = (g.p == 2) ? t1 * g.L + t2 : t1;
        if (t < s) continue;
        hcb[(size_t)s * (b + 1) + (t - s)] = nb[(size_t)s * nn + k];
      }
    }
    DD_CUDA(cudaMemcpyAsync(CB, hcb.data(), cb, cudaMemcpyHostToDevice, c->stream));
    launch_band_factor(c, CB, RB, inv, 1, N, b, flag, nullptr);
    if (!c->A0inv) c->A0inv = (double*)dev_alloc(c, sizeof(double) * (size_t)N * N);
    launch_band_inverse_rows(N, b, CB, RB, inv, c->A0inv, c->stream);
  }
  int fl = 0;
  DD_CUDA(cudaMemcpyAsync(&fl, flag, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  DD_CUDA(cudaStreamSynchronize(c->stream));
  if (fl) throw Error(DD_ENOTSPD, "coarse matrix A_0 not positive definite");
  return DD_OK;
}

// c_i = (D_i R_i psi)^T r, block per subdomain
__global__ void k_coarse_restrict(Geo g, const Sub* __restrict__ subs, const double* __restrict__ wT, int kpad,
                                  const double* __restrict__ r, double* __restrict__ c0, const PcgState* st) {
  if (st != nullptr && st->done) return;
  const int s = blockIdx.x;
  const Sub sb = subs[s];
  double acc[1] = {0.0};
  for (int k = threadIdx.x; k < sb.nloc; k += blockDim.x)
    acc[0] = fma(wT[(size_t)sb.type * kpad + loc_pad(g, k)], r[sub_global(g, sb, k)], acc[0]);
  block_sum<1>(acc);
  if (threadIdx.x == 0) c0[s] = acc[0];
}

void launch_coarse_restrict(dd_ctx* c, const double* r, cudaStream_t s) {
  (k_coarse_restrict<<<c->g.nsub, 256, 0, s>>>(c->g, c->subs, c->wT, c->kpad, r, c->c0, c->st), dd::note_launch());
  DD_CUDA(cudaGetLastError());
}

void launch_coarse_solve(dd_ctx* c, cudaStream_t s) {
  const Geo& g = c->g;
  if (!c->coarse_dense) {
    const size_t W2 = (size_t)c->cr_w2, ncoef = 2 * (size_t)c->cr_c2 + 3 * W2;
    const size_t full = sizeof(double) * (W2 + ncoef);   // f + coefficients
    const int staged = full <= 200 * 1024 ? 1 : 0;
    const size_t smem = staged ? full : sizeof(double) * W2;
    if (smem > 220 * 1024) throw Error(DD_EINVAL, "coarse chain too long for the shared-memory cyclic reduction");
    static PerDeviceOnce attr;   // once per device
    once_per_device(attr, [] {
      DD_CUDA(cudaFuncSetAttribute(k_cr_solve, cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024));
    });
    (k_cr_solve<<<1, kCrThreads, smem, s>>>(c->cr, g.nsub, c->cr_m, c->cr_c2, c->cr_w2, c->c0, c->u0, c->u0f, c->st,
                                             staged, c->dev_err + 8),
     dd::note_launch());
  } else {
    const int N = g.nsub;
    (k_gemv_rows<<<(N + 7) / 8, 256, 0, s>>>(N, c->A0inv, c->c0, c->u0, c->u0f, c->st), dd::note_launch());
  }
  DD_CUDA(cudaGetLastError());
}

void launch_b_cr_solve(const BInst* B, int n, size_t smem, cudaStream_t s) {
  static PerDeviceOnce attr;   // once per device
  once_per_device(attr, [] {
    DD_CUDA(cudaFuncSetAttribute(kb_cr_solve, cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024));
  });
  (kb_cr_solve<<<n, kCrThreads, smem, s>>>(B), dd::note_launch());
  DD_CUDA(cudaGetLastError());
}

// shared memory and staging of the plain p = 1 coarse solve of one context (cyclic reduction)
void cr_launch_shape(const dd_ctx* c, size_t* smem, int* staged) {
  const size_t W2 = (size_t)c->cr_w2, ncoef = 2 * (size_t)c->cr_c2 + 3 * W2;
  const size_t full = sizeof(double) * (W2 + ncoef);
  *staged = full <= 200 * 1024 ? 1 : 0;
  *smem = *staged ? full : sizeof(double) * W2;
}

}  // namespace dd
