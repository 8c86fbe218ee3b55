// Local subdomain matrices and their banded Cholesky factors; the FP64 local solves of
// the plain method; the cell eigenpair.
//
// Local problems (Sec. 3.1): A_{sigma,i} = R_i A_sigma R_i^T on the interior nodes strictly
// inside the open overlapping box Omega_i (homogeneous Dirichlet on its artificial
// boundary).  All subdomains with the same clipping (left / interior / right per axis) have
// identical matrices, because the cells are translated copies and V is periodic (A1); the
// factors are stored once per type.  Local order: (c1, c2, j) with j fastest, so the
// half bandwidth is nyi + 1 (p = 1) or w2 nyi + nyi + 1 (p = 2).
#include <atomic>

#include "dd_band.cuh"

namespace dd {

// ----------------------------------------------------------------------------------------
// Banded Cholesky A = L L^T, one CTA per matrix, right-looking.  Input: the lower band of A
// in CB (CB[i][d] = A(i+d, i)).  Output in place: CB[i][d] = L(i+d, i)/L(i, i) (d >= 1),
// CB[i][0] = L(i, i), inv[i] = 1/L(i, i)^2 (the storage the band solves expect).
// A zero or negative pivot sets *flag (DD_ENOTSPD) and continues with pivot 1.
//
// k_band_factor_win keeps the active (b+1) x (b+1) window in shared memory as a ring of
// columns: every column is read from global memory once and written back once when it is
// final, so each step waits on shared memory only.  k_band_factor (global window) serves
// bandwidths whose window does not fit.
// ----------------------------------------------------------------------------------------
constexpr int kBandWinMax = 160;
constexpr int kMaxPairs = 16;   // triangle pairs per thread: b (b + 1) / 2 <= 16 x threads for b <= 160

template <int P>
__global__ void __launch_bounds__(1024) k_band_factor_win(double* CB, double* inv, const int* __restrict__ nvec,
                                                          int nmax, int b, int* flag) {
  extern __shared__ double fsm[];
  const int m = blockIdx.x;
  const int n = nvec[m];
  const int bs = b + 1, W = b + 1;
  const int t = threadIdx.x;   // owns entry d = t of the columns it stages (bs <= blockDim.x)
  double* win = fsm;               // W columns x bs entries
  double* colk = fsm + W * bs;     // L(k+d, k), d = 0..b
  double* A = CB + (size_t)m * nmax * bs;
  double* iv = inv + (size_t)m * nmax;
  // this thread's pairs (d1, d2), 1 <= d2 <= d1 <= b, of the lower triangle of the window
  // update: linear index e = d1 (d1 - 1) / 2 + d2 - 1 taken as e = t, t + T, ...; in that order
  // d1 never decreases, so the pairs beyond the last column's reach form a suffix
  unsigned pr[kMaxPairs / 2];   // two pairs per word: (d1 << 8 | d2) in each half (b <= 160 < 256)
  int npr = 0;
  {
    const int T = (int)blockDim.x, tot = b * (b + 1) / 2;
#pragma unroll
    for (int j = 0; j < kMaxPairs; ++j) {
      const int e = t + j * T;
      int d1 = 0, d2 = 0;
      if (e < tot) {
        d1 = (int)((sqrtf(8.0f * (float)e + 1.0f) + 1.0f) * 0.5f);   // first guess, then exact
        while (d1 * (d1 - 1) / 2 > e) --d1;
        while ((d1 + 1) * d1 / 2 <= e) ++d1;
        d2 = e - d1 * (d1 - 1) / 2 + 1;
        ++npr;
      }
      const unsigned half = ((unsigned)d1 << 8) | (unsigned)d2;
      if (j & 1) pr[j >> 1] |= half << 16;
      else pr[j >> 1] = half;
    }
  }
  const int first = min(W, n);
  for (int e = t; e < first * bs; e += blockDim.x) win[e] = A[e];
  // entering columns are loaded P steps before they are needed
  double ring[P];
#pragma unroll
  for (int u = 0; u < P; ++u) {
    const int j = W + u;
    ring[u] = A[(size_t)min(j, n - 1) * bs + min(t, b)];   // clamped: no select on the load
  }
  __syncthreads();
  for (int k0 = 0; k0 < n; k0 += P) {
#pragma unroll
    for (int u = 0; u < P; ++u) {
      const int k = k0 + u;
      if (k < n) {
        const int sk = k % W;
        if (t == 0) {
          double piv = win[sk * bs];
          if (!(piv > 0.0)) {
            atomicOr(flag, 1);
            piv = 1.0;
          }
          const double il = rsqrt(piv);
          A[(size_t)k * bs] = piv * il;
          iv[k] = il * il;
          colk[0] = il;
        }
        __syncthreads();
        const double il = colk[0];
        const int dmax = min(b, n - 1 - k);
        for (int d = 1 + t; d <= b; d += blockDim.x) {
          double v = 0.0;
          if (d <= dmax) {
            v = win[sk * bs + d] * il;           // L(k+d, k)
            A[(size_t)k * bs + d] = v * il;      // pre-scaled by 1/L(k,k)
          }
          colk[d] = v;
        }
        __syncthreads();
        // A(k+d1, k+d2) -= L(k+d1, k) L(k+d2, k) over this thread's pairs with d1 <= dmax
#pragma unroll
        for (int j = 0; j < kMaxPairs; ++j) {
          const unsigned half = (j & 1) ? (pr[j >> 1] >> 16) : (pr[j >> 1] & 0xFFFFu);
          const int d1 = (int)(half >> 8), d2 = (int)(half & 0xFFu);
          if (j < npr && d1 <= dmax) {
            int slot = sk + d2;                  // ring slot of column k + d2
            if (slot >= W) slot -= W;
            double* a = win + slot * bs + (d1 - d2);
            *a = fma(-colk[d1], colk[d2], *a);
          }
        }
        __syncthreads();
        // the slot of column k is free: store column k + W (untouched so far), prefetch k + W + P
        if (k + W < n && t < bs) win[sk * bs + t] = ring[u];
        const int j = k + W + P;
        ring[u] = A[(size_t)min(j, n - 1) * bs + min(t, b)];
      }
    }
  }
}

__global__ void __launch_bounds__(1024) k_band_factor(double* CB, double* inv, const int* __restrict__ nvec,
                                                      int nmax, int b, int* flag) {
  extern __shared__ double colk[];
  const int m = blockIdx.x;
  const int n = nvec[m];
  const int bs = b + 1;
  double* A = CB + (size_t)m * nmax * bs;
  double* iv = inv + (size_t)m * nmax;
  for (int k = 0; k < n; ++k) {
    if (threadIdx.x == 0) {
      double piv = A[(size_t)k * bs];
      if (!(piv > 0.0)) {
        atomicOr(flag, 1);
        piv = 1.0;
      }
      const double l = sqrt(piv);
      A[(size_t)k * bs] = l;
      iv[k] = 1.0 / piv;
      colk[0] = 1.0 / l;
    }
    __syncthreads();
    const double il = colk[0];
    const int dmax = min(b, n - 1 - k);
    for (int d = 1 + threadIdx.x; d <= b; d += blockDim.x) {
      double v = 0.0;
      if (d <= dmax) v = A[(size_t)k * bs + d] * il;
      colk[d] = v;
    }
    __syncthreads();
    // A(k+d1, k+d2) -= L(k+d1,k) L(k+d2,k), 1 <= d2 <= d1 <= dmax; stored at CB[k+d2][d1-d2]
    const int tot = dmax * dmax;
    for (int t = threadIdx.x; t < tot; t += blockDim.x) {
      const int d1 = t / dmax + 1, d2 = t % dmax + 1;
      if (d2 <= d1) {
        double* a = A + (size_t)(k + d2) * bs + (d1 - d2);
        *a = fma(-colk[d1], colk[d2], *a);
      }
    }
    for (int d = 1 + threadIdx.x; d <= dmax; d += blockDim.x) A[(size_t)k * bs + d] = colk[d] * il;
    __syncthreads();
  }
}

// launch the factorisation of nmat band matrices (sizes in nvec) and build the row band
static void factor_launch(const Geo&, double* CB, double* RB, double* inv, const int* nvec, int nmat, int nmax, int b,
                          int* flag, cudaStream_t s);

// RB[i][d] = L(i, i-d) = CB[i-d][d]
__global__ void k_band_rows(const double* __restrict__ CB, double* RB, const int* __restrict__ nvec,
                            int nmat, int nmax, int b) {
  const int bs = b + 1;
  const long long total = (long long)nmat * nmax * bs;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const int m = (int)(t / ((long long)nmax * bs));
    const long long rem = t - (long long)m * nmax * bs;
    const int i = (int)(rem / bs), d = (int)(rem % bs);
    const int n = nvec[m];
    double v = 0.0;
    if (i < n && i - d >= 0) v = CB[((size_t)m * nmax + (i - d)) * bs + d];
    RB[t] = v;
  }
}

int launch_band_factor(dd_ctx* c, double* CB, double* RB, double* inv, int nmat, int nmax, int b, int* flag) {
  // nvec: sizes of the matrices, taken from ctx scratch (c->dev_err + 16 ...) -> use a temp
  int* nvec = nullptr;
  DD_CUDA(cudaMallocAsync(&nvec, sizeof(int) * nmat, c->stream));
  std::vector<int> nh(nmat);
  if (CB == c->bandCB) {
    for (int t = 0; t < nmat; ++t) nh[t] = c->type_nloc[t];
  } else {
    for (int t = 0; t < nmat; ++t) nh[t] = nmax;
  }
  DD_CUDA(cudaMemcpyAsync(nvec, nh.data(), sizeof(int) * nmat, cudaMemcpyHostToDevice, c->stream));
  factor_launch(c->g, CB, RB, inv, nvec, nmat, nmax, b, flag, c->stream);
  DD_CUDA(cudaFreeAsync(nvec, c->stream));
  return DD_OK;
}

static void factor_launch(const Geo&, double* CB, double* RB, double* inv, const int* nvec, int nmat, int nmax, int b,
                          int* flag, cudaStream_t s) {
  if (b <= kBandWinMax) {
    const size_t smem = sizeof(double) * ((size_t)(b + 1) * (b + 1) + (b + 1));
    const int tot = b * (b + 1) / 2;   // triangle pairs: at most kMaxPairs per thread
    const int threads = (b * b > 2048) ? (tot > kMaxPairs * 512 ? 1024 : 512) : 256;
    static std::atomic<bool> attr{false};   // set once per process (idempotent if two threads race)
    if (!attr) {
      DD_CUDA(cudaFuncSetAttribute(k_band_factor_win<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024));
      attr = true;
    }
    (k_band_factor_win<4><<<nmat, threads, smem, s>>>(CB, inv, nvec, nmax, b, flag), dd::note_launch());
  } else {
    (k_band_factor<<<nmat, 1024, sizeof(double) * (b + 1), s>>>(CB, inv, nvec, nmax, b, flag), dd::note_launch());
  }
  DD_CUDA(cudaGetLastError());
  const long long total = (long long)nmat * nmax * (b + 1);
  (k_band_rows<<<grid_blocks(total, kThreads), kThreads, 0, s>>>(CB, RB, nvec, nmat, nmax, b), dd::note_launch());
  DD_CUDA(cudaGetLastError());
}

// ----------------------------------------------------------------------------------------
// Local matrix assembly from the A_sigma stencil table: CB[t][k][k'-k] = A_sigma(k', k), k' >= k.
// ----------------------------------------------------------------------------------------
__global__ void k_local_assemble(Geo g, const double* __restrict__ tabS, const Sub* __restrict__ rep,
                                 int ntypes, int nmax, int b, double* CB) {
  const int bs = b + 1;
  const long long total = (long long)ntypes * nmax;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const int ty = (int)(t / nmax);
    const int k = (int)(t - (long long)ty * nmax);
    const Sub s = rep[ty];
    if (k >= s.nloc) continue;
    const int sj = k % g.nyi;
    const int cc = k / g.nyi;
    const int c1 = cc / s.w2, c2 = cc % s.w2;
    const int a1 = s.lo1 + c1, a2 = s.lo2 + c2;
    int cls;
    if (g.p == 1) cls = (a1 % g.n) * g.Ypad + sj;
    else cls = ((a1 % g.n) * g.n + (a2 % g.n)) * g.Ypad + sj;
    double* row = CB + ((size_t)ty * nmax + k) * bs;
    for (int tap = 0; tap < g.ntap; ++tap) {
      int d1, d2 = 0, dy;
      if (g.p == 1) { d1 = tap / 3 - 1; dy = tap % 3 - 1; }
      else { d1 = tap / 9 - 1; d2 = (tap / 3) % 3 - 1; dy = tap % 3 - 1; }
      const int n1 = c1 + d1, n2 = c2 + d2, nj = sj + dy;
      if (n1 < 0 || n1 >= s.w1 || n2 < 0 || n2 >= s.w2 || nj < 0 || nj >= g.nyi) continue;
      const int kk = (n1 * s.w2 + n2) * g.nyi + nj;
      if (kk < k) continue;
      row[kk - k] = tabS[(size_t)tap * g.ncls + cls];
    }
  }
}

void launch_local_assemble(dd_ctx* c) {
  // representative subdomain of every type
  std::vector<Sub> rep(c->ntypes);
  for (int t = 0; t < c->ntypes; ++t) {
    for (const Sub& s : c->subs_h)
      if (s.type == t) { rep[t] = s; break; }
  }
  Sub* drep = nullptr;
  DD_CUDA(cudaMallocAsync(&drep, sizeof(Sub) * c->ntypes, c->stream));
  DD_CUDA(cudaMemcpyAsync(drep, rep.data(), sizeof(Sub) * c->ntypes, cudaMemcpyHostToDevice, c->stream));
  const size_t nbytes = sizeof(double) * (size_t)c->ntypes * c->nloc_max * (c->band + 1);
  DD_CUDA(cudaMemsetAsync(c->bandCB, 0, nbytes, c->stream));
  const long long total = (long long)c->ntypes * c->nloc_max;
  (k_local_assemble<<<grid_blocks(total, 128), 128, 0, c->stream>>>(c->g, c->tabS, drep, c->ntypes,
                                                                   c->nloc_max, c->band, c->bandCB), dd::note_launch());
  DD_CUDA(cudaGetLastError());
  DD_CUDA(cudaFreeAsync(drep, c->stream));
}

// ----------------------------------------------------------------------------------------
// FP64 local solves y_i = A_{sigma,i}^{-1} R_i r for every subdomain (one warp each); the
// result goes to Y[slot(i)][k]; the prolong-sum gathers it.
// ----------------------------------------------------------------------------------------
template <int NV, int PF, int K>
__global__ void k_local_solve(Geo g, const Sub* __restrict__ subs, const int2* __restrict__ groups, int ngroups,
                              const int* __restrict__ sub_of_slot, const double* __restrict__ r,
                              const double* __restrict__ CB, const double* __restrict__ RB,
                              const double* __restrict__ inv, int nmax, int b, double* __restrict__ Y, int kpad,
                              const double* __restrict__ wT, double* c0, const PcgState* st) {
  if (st != nullptr && st->done) return;
  extern __shared__ double xs_all[];
  const int wpb = blockDim.x >> 5;
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int gi = blockIdx.x * wpb + wid;
  if (gi >= ngroups) return;
  const int2 grp = groups[gi];   // K (or fewer) consecutive slots of one type
  constexpr int RING = band_ring_doubles<NV, PF>();
  double* xs = xs_all + (size_t)wid * (K * nmax + RING);
  double* ring = xs + (size_t)K * nmax;
  const int type = subs[sub_of_slot[grp.x]].type;
  int n = 0;
#pragma unroll
  for (int j = 0; j < K; ++j) {
    double* xj = xs + (size_t)j * nmax;
    if (j < grp.y) {
      const int s = sub_of_slot[grp.x + j];
      const Sub sb = subs[s];
      n = sb.nloc;
      // gather R_i r; the coarse right-hand side (D_i R_i psi)^T r rides along (Def. 2.1)
      double cr = 0.0;
      const double* wt = wT + (size_t)type * kpad;
      for (int k = lane; k < sb.nloc; k += 32) {
        const int sj = k % g.nyi, cc = k / g.nyi;
        const int c1 = cc / sb.w2, c2 = cc % sb.w2;
        long long idx;
        if (g.p == 1) idx = (long long)(sb.lo1 + c1) * g.Ypad + sj;
        else idx = ((long long)(sb.lo1 + c1) * g.ncx + (sb.lo2 + c2)) * g.Ypad + sj;
        const double v = r[idx];
        xj[k] = v;
        if (c0 != nullptr) cr = fma(wt[k], v, cr);
      }
      if (c0 != nullptr) {
        cr = warp_sum(cr);
        if (lane == 0) c0[s] = cr;
      }
    } else {
      for (int k = lane; k < nmax; k += 32) xj[k] = 0.0;
    }
  }
  const size_t off = (size_t)type * nmax;
  band_solve_k<NV, PF, K>(xs, nmax, n, b, CB + off * (b + 1), RB + off * (b + 1), inv + off, ring);
  __syncwarp();
  for (int j = 0; j < grp.y; ++j) {
    double* y = Y + (size_t)(grp.x + j) * kpad;
    for (int k = lane; k < n; k += 32) y[k] = xs[(size_t)j * nmax + k];
  }
}

void launch_band_solve_local(dd_ctx* c, const double* r, double* c0, cudaStream_t s) {
  const int K = c->rhs_k;
  const int wpb = 1;
  const size_t smem = sizeof(double) * (size_t)K * c->nloc_max + band_ring_bytes(c->band);
  const int nb = c->ngroups;
  DD_BAND_DISPATCH(c->band, {
    DD_K_DISPATCH(K, {
      constexpr int KK = (NV == 0 || NV > 4) ? 1 : KR;
      if (K > KK) throw Error(DD_EINVAL, "local right-hand sides per warp exceed the kernel's");
      static std::atomic<bool> attr_set{false};
      if (!attr_set) {
        DD_CUDA(cudaFuncSetAttribute(k_local_solve<NV, PF, KK>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     220 * 1024));
        attr_set = true;
      }
      (k_local_solve<NV, PF, KK><<<nb, wpb * 32, smem, s>>>(c->g, c->subs, c->groups, c->ngroups, c->sub_of_slot,
                                                           r, c->bandCB, c->bandRB, c->bandInv, c->nloc_max,
                                                           c->band, c->Y64, c->kpad, c->wT, c0, c->st),
       dd::note_launch());
    });
  });
  DD_CUDA(cudaGetLastError());
}

// ----------------------------------------------------------------------------------------
// Cell eigenpair (cell problem of Sec. 1 / weak cell problem of Sec. 2): lowest eigenpair of
// A_# psi = sigma M_# psi with x-periodic, y-Dirichlet conditions, by shifted inverse
// iteration with shift s = min V - 1 (A_# - s M_# is SPD because M_V >= min(V) M for a
// quadrature with positive weights).  The factor uses an interleaved x order
// (0, n-1, 1, n-2, ...) that keeps periodic neighbours within two positions, so the
// periodic operator is banded.
// ----------------------------------------------------------------------------------------
__host__ __device__ inline int ipos(int a, int n) { return (2 * a < n) ? 2 * a : 2 * (n - 1 - a) + 1; }

__global__ void __launch_bounds__(1024) k_cell_shift(const double* __restrict__ V, long long nV, double* shift) {
  double m = 1e300;
  for (long long t = threadIdx.x; t < nV; t += blockDim.x) m = fmin(m, V[t]);
  __shared__ double sm[32];
  for (int o = 16; o > 0; o >>= 1) m = fmin(m, __shfl_down_sync(kFull, m, o));
  if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    double v = sm[0];
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) v = fmin(v, sm[w]);
    *shift = v - 1.0;
  }
}

// cell DOF (natural) k = (a1 [n + a2]) nyi + sj; interleaved row ri = (ipos(a1) [n + ipos(a2)]) nyi + sj
__global__ void k_cell_assemble(Geo g, const double* __restrict__ tabA, const double* __restrict__ tabM,
                                const double* __restrict__ shift, int b, double* CB) {
  const int bs = b + 1;
  const int ncol = (g.p == 1) ? g.n : g.n * g.n;
  const long long ncell = (long long)ncol * g.nyi;
  const double s = *shift;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < ncell;
       t += (long long)gridDim.x * blockDim.x) {
    const int sj = (int)(t % g.nyi);
    const int cc = (int)(t / g.nyi);
    int a1, a2 = 0, cls, row;
    if (g.p == 1) {
      a1 = cc;
      cls = a1 * g.Ypad + sj;
      row = ipos(a1, g.n) * g.nyi + sj;
    } else {
      a1 = cc / g.n;
      a2 = cc % g.n;
      cls = (a1 * g.n + a2) * g.Ypad + sj;
      row = (ipos(a1, g.n) * g.n + ipos(a2, g.n)) * g.nyi + sj;
    }
    for (int tap = 0; tap < g.ntap; ++tap) {
      int d1, d2 = 0, dy;
      if (g.p == 1) { d1 = tap / 3 - 1; dy = tap % 3 - 1; }
      else { d1 = tap / 9 - 1; d2 = (tap / 3) % 3 - 1; dy = tap % 3 - 1; }
      const int nj = sj + dy;
      if (nj < 0 || nj >= g.nyi) continue;
      const int b1 = (a1 + d1 + g.n) % g.n;
      int col;
      if (g.p == 1) col = ipos(b1, g.n) * g.nyi + nj;
      else {
        const int b2 = (a2 + d2 + g.n) % g.n;
        col = (ipos(b1, g.n) * g.n + ipos(b2, g.n)) * g.nyi + nj;
      }
      if (col < row) continue;
      const size_t ti = (size_t)tap * g.ncls + cls;
      CB[(size_t)row * bs + (col - row)] += tabA[ti] - s * tabM[ti];
    }
  }
}

// periodic cell stencil y = T x (natural cell order), CTA-wide
__device__ void cell_stencil(const Geo& g, const double* __restrict__ tab, const double* x, double* y, int ncell) {
  for (int k = threadIdx.x; k < ncell; k += blockDim.x) {
    const int sj = k % g.nyi, cc = k / g.nyi;
    int a1, a2 = 0, cls;
    if (g.p == 1) { a1 = cc; cls = a1 * g.Ypad + sj; }
    else { a1 = cc / g.n; a2 = cc % g.n; cls = (a1 * g.n + a2) * g.Ypad + sj; }
    double acc = 0.0;
    for (int tap = 0; tap < g.ntap; ++tap) {
      int d1, d2 = 0, dy;
      if (g.p == 1) { d1 = tap / 3 - 1; dy = tap % 3 - 1; }
      else { d1 = tap / 9 - 1; d2 = (tap / 3) % 3 - 1; dy = tap % 3 - 1; }
      const int nj = sj + dy;
      if (nj < 0 || nj >= g.nyi) continue;
      const int b1 = (a1 + d1 + g.n) % g.n;
      int kk;
      if (g.p == 1) kk = b1 * g.nyi + nj;
      else kk = (b1 * g.n + (a2 + d2 + g.n) % g.n) * g.nyi + nj;
      acc = fma(__ldg(tab + (size_t)tap * g.ncls + cls), x[kk], acc);
    }
    y[k] = acc;
  }
}

template <int NV>
__device__ void cta_sum(double (&v)[NV]) {   // result broadcast to every thread
  __shared__ double res[NV];
  block_sum<NV>(v);
  if (threadIdx.x == 0)
    for (int k = 0; k < NV; ++k) res[k] = v[k];
  __syncthreads();
  for (int k = 0; k < NV; ++k) v[k] = res[k];
  __syncthreads();
}

struct CellOut {
  double sigma, eta, drho, shift;
  int iters, status;
};

constexpr int kCellThreads = 512;

// ---- cell inverse iteration on a dense inverse -------------------------------------------
// G = (A_# - s M_#)^{-1} is formed once per shift from the band factor (every column an
// independent band solve, one warp each, all in parallel) and permuted to the natural cell
// order; each inverse-iteration step is then y = M_# x (stencil), w = G y (a GEMV across the
// GPU) and one CTA that normalises, forms rho and eta and applies the stop rule.  The state
// lives on the device; the host reads it every few steps.
struct CellState {
  double rho, rho_prev, eta, eta_prev, drho;
  int iters, stable, done, status;
};

__global__ void k_cell_perm_dense(Geo g, int ncell, const double* __restrict__ Gi, double* __restrict__ Gn) {
  // Gn[i][j] = Gi[pos(i)][pos(j)], natural index k = (a1 [n + a2]) nyi + sj
  const long long total = (long long)ncell * ncell;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(t / ncell), j = (int)(t % ncell);
    int pi, pj;
    {
      const int sj = i % g.nyi, cc = i / g.nyi;
      pi = (g.p == 1) ? ipos(cc, g.n) * g.nyi + sj : (ipos(cc / g.n, g.n) * g.n + ipos(cc % g.n, g.n)) * g.nyi + sj;
    }
    {
      const int sj = j % g.nyi, cc = j / g.nyi;
      pj = (g.p == 1) ? ipos(cc, g.n) * g.nyi + sj : (ipos(cc / g.n, g.n) * g.n + ipos(cc % g.n, g.n)) * g.nyi + sj;
    }
    Gn[t] = Gi[(size_t)pi * ncell + pj];
  }
}

// y = M_# x over the cell, grid-wide
__global__ void k_cell_mass(Geo g, int ncell, const double* __restrict__ tabM, const double* __restrict__ x,
                            double* __restrict__ y, const CellState* cs) {
  if (cs->done) return;
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < ncell; k += gridDim.x * blockDim.x) {
    const int sj = k % g.nyi, cc = k / g.nyi;
    int a1, a2 = 0, cls;
    if (g.p == 1) { a1 = cc; cls = a1 * g.Ypad + sj; }
    else { a1 = cc / g.n; a2 = cc % g.n; cls = (a1 * g.n + a2) * g.Ypad + sj; }
    double acc = 0.0;
    for (int tap = 0; tap < g.ntap; ++tap) {
      int d1, d2 = 0, dy;
      if (g.p == 1) { d1 = tap / 3 - 1; dy = tap % 3 - 1; }
      else { d1 = tap / 9 - 1; d2 = (tap / 3) % 3 - 1; dy = tap % 3 - 1; }
      const int nj = sj + dy;
      if (nj < 0 || nj >= g.nyi) continue;
      const int b1 = (a1 + d1 + g.n) % g.n;
      const int kk = (g.p == 1) ? b1 * g.nyi + nj : (b1 * g.n + (a2 + d2 + g.n) % g.n) * g.nyi + nj;
      acc = fma(__ldg(tabM + (size_t)tap * g.ncls + cls), x[kk], acc);
    }
    y[k] = acc;
  }
}

// w = G y, warp per row
__global__ void k_cell_gemv(int n, const double* __restrict__ G, const double* __restrict__ y, double* __restrict__ w,
                            const CellState* cs) {
  if (cs->done) return;
  const int lane = threadIdx.x & 31;
  const int row = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (row >= n) return;
  const double* gr = G + (size_t)row * n;
  double acc = 0.0;
  for (int k = lane; k < n; k += 32) acc = fma(gr[k], y[k], acc);
  acc = warp_sum(acc);
  if (lane == 0) w[row] = acc;
}

// x = w / ||w||_M (sign: sum > 0), rho = x^T A_# x, eta = ||A x - rho M x|| / (|rho| ||M x||), stop rule
__global__ void __launch_bounds__(kCellThreads) k_cell_update(Geo g, int ncell, const double* __restrict__ tabA,
                                                             const double* __restrict__ tabM, const double* w,
                                                             double* x, double tol_drho, double tol_eta, int maxit,
                                                             CellState* cs) {
  if (cs->done) return;
  extern __shared__ double sm[];
  double* xs = sm;            // w, then x
  double* ys = sm + ncell;    // M x
  double* zs = sm + 2 * ncell;
  for (int k = threadIdx.x; k < ncell; k += blockDim.x) xs[k] = w[k];
  __syncthreads();
  cell_stencil(g, tabM, xs, ys, ncell);
  __syncthreads();
  double d2[2] = {0.0, 0.0};
  for (int k = threadIdx.x; k < ncell; k += blockDim.x) {
    d2[0] = fma(xs[k], ys[k], d2[0]);
    d2[1] += xs[k];
  }
  cta_sum<2>(d2);
  if (!(d2[0] > 0.0)) {
    if (threadIdx.x == 0) { cs->status = DD_ENAN; cs->done = 1; }
    return;
  }
  const double sc = (d2[1] < 0.0 ? -1.0 : 1.0) / sqrt(d2[0]);
  for (int k = threadIdx.x; k < ncell; k += blockDim.x) {
    xs[k] *= sc;
    ys[k] *= sc;
  }
  __syncthreads();
  cell_stencil(g, tabA, xs, zs, ncell);
  __syncthreads();
  double d1[1] = {0.0};
  for (int k = threadIdx.x; k < ncell; k += blockDim.x) d1[0] = fma(xs[k], zs[k], d1[0]);
  cta_sum<1>(d1);
  const double rho = d1[0];
  double d3[2] = {0.0, 0.0};
  for (int k = threadIdx.x; k < ncell; k += blockDim.x) {
    const double e = fma(-rho, ys[k], zs[k]);
    d3[0] = fma(e, e, d3[0]);
    d3[1] = fma(ys[k], ys[k], d3[1]);
  }
  cta_sum<2>(d3);
  for (int k = threadIdx.x; k < ncell; k += blockDim.x) x[k] = xs[k];
  if (threadIdx.x == 0) {
    const double eta = sqrt(d3[0] / d3[1]) / fabs(rho);
    const double drho = fabs(rho - cs->rho_prev);
    cs->iters += 1;
    cs->rho = rho;
    cs->eta = eta;
    cs->drho = drho;
    if (!isfinite(rho)) {
      cs->status = DD_ENAN;
      cs->done = 1;
    } else {
      // at the residual target, stop once the Rayleigh quotient is stationary or the residual
      // no longer improves (its rounding floor grows as the shift nears sigma_1)
      if (eta <= tol_eta && (drho <= tol_drho * fabs(rho) || eta >= 0.5 * cs->eta_prev)) cs->stable += 1;
      else cs->stable = 0;
      if (cs->stable >= 2) cs->done = 1;
      else if (cs->iters >= maxit) {
        cs->status = DD_EMAXIT;
        cs->done = 1;
      }
    }
    cs->eta_prev = eta;
    cs->rho_prev = rho;
  }
}

// one phase of the cell solve: assemble A_# - s M_#, factor, invert, iterate; returns false
// if the factorisation met a non-positive pivot (s not below sigma_1)
static bool cell_phase(dd_ctx* c, double* shift, bool from_minV, double margin_frac, int warm, double tol_drho,
                       double tol_eta, int maxit, CellOut* out_h) {
  const Geo& g = c->g;
  const int ncell = (int)c->ncell;
  const int b = c->cell_band;
  const size_t cbsz = sizeof(double) * (size_t)ncell * (b + 1);
  const size_t gsz = sizeof(double) * (size_t)ncell * ncell;
  double *CB = nullptr, *RB = nullptr, *inv = nullptr, *Gi = nullptr, *Gn = nullptr, *y = nullptr, *w = nullptr;
  CellState* cs = nullptr;
  int* flag = c->dev_err + 1;
  int* nvec = nullptr;
  DD_CUDA(cudaMallocAsync(&CB, cbsz, c->stream));
  DD_CUDA(cudaMallocAsync(&RB, cbsz, c->stream));
  DD_CUDA(cudaMallocAsync(&inv, sizeof(double) * ncell, c->stream));
  DD_CUDA(cudaMallocAsync(&nvec, sizeof(int), c->stream));
  DD_CUDA(cudaMemsetAsync(CB, 0, cbsz, c->stream));
  DD_CUDA(cudaMemsetAsync(flag, 0, sizeof(int), c->stream));
  DD_CUDA(cudaMemcpyAsync(nvec, &ncell, sizeof(int), cudaMemcpyHostToDevice, c->stream));
  if (from_minV) {
    long long nV = (long long)((g.p == 1) ? g.n : g.n * g.n) * g.ny;
    for (int k = 0; k <= g.p; ++k) nV *= g.Q;
    (k_cell_shift<<<1, 1024, 0, c->stream>>>(c->Vqp, nV, shift), dd::note_launch());
  } else {
    // shift = rho - margin_frac (rho - s_previous), from the previous phase's result
    const double s_new = out_h->sigma - margin_frac * (out_h->sigma - out_h->shift);
    DD_CUDA(cudaMemcpyAsync(shift, &s_new, sizeof(double), cudaMemcpyHostToDevice, c->stream));
  }
  (k_cell_assemble<<<grid_blocks(ncell, 128), 128, 0, c->stream>>>(g, c->tabA, c->tabM, shift, b, CB), dd::note_launch());
  factor_launch(g, CB, RB, inv, nvec, 1, ncell, b, flag, c->stream);
  int fl = 0;
  DD_CUDA(cudaMemcpyAsync(&fl, flag, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  DD_CUDA(cudaStreamSynchronize(c->stream));
  bool ok = (fl == 0);
  if (ok) {
    DD_CUDA(cudaMallocAsync(&Gi, gsz, c->stream));
    DD_CUDA(cudaMallocAsync(&Gn, gsz, c->stream));
    DD_CUDA(cudaMallocAsync(&y, sizeof(double) * ncell, c->stream));
    DD_CUDA(cudaMallocAsync(&w, sizeof(double) * ncell, c->stream));
    DD_CUDA(cudaMallocAsync(&cs, sizeof(CellState), c->stream));
    launch_band_inverse_rows(ncell, b, CB, RB, inv, Gi, c->stream);
    (k_cell_perm_dense<<<grid_blocks((long long)ncell * ncell, kThreads), kThreads, 0, c->stream>>>(g, ncell, Gi, Gn),
     dd::note_launch());
    CellState init{};
    init.rho_prev = 1e300;
    init.eta_prev = 1e300;
    DD_CUDA(cudaMemcpyAsync(cs, &init, sizeof(init), cudaMemcpyHostToDevice, c->stream));
    if (!warm) {
      std::vector<double> ones((size_t)ncell, 1.0);
      DD_CUDA(cudaMemcpyAsync(c->psi_cell, ones.data(), sizeof(double) * ncell, cudaMemcpyHostToDevice, c->stream));
      DD_CUDA(cudaStreamSynchronize(c->stream));
    }
    const size_t smem = sizeof(double) * 3 * (size_t)ncell;
    DD_CUDA(cudaFuncSetAttribute(k_cell_update, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const int gemv_blocks = (ncell + 7) / 8;
    CellState h{};
    for (int it = 0; it < maxit; it += 4) {
      for (int k = 0; k < 4; ++k) {
        (k_cell_mass<<<grid_blocks(ncell, 256), 256, 0, c->stream>>>(g, ncell, c->tabM, c->psi_cell, y, cs),
         dd::note_launch());
        (k_cell_gemv<<<gemv_blocks, 256, 0, c->stream>>>(ncell, Gn, y, w, cs), dd::note_launch());
        (k_cell_update<<<1, kCellThreads, smem, c->stream>>>(g, ncell, c->tabA, c->tabM, w, c->psi_cell, tol_drho,
                                                           tol_eta, maxit, cs), dd::note_launch());
      }
      DD_CUDA(cudaGetLastError());
      DD_CUDA(cudaMemcpyAsync(&h, cs, sizeof(CellState), cudaMemcpyDeviceToHost, c->stream));
      DD_CUDA(cudaStreamSynchronize(c->stream));
      if (h.done) break;
    }
    double sh = 0.0;
    DD_CUDA(cudaMemcpyAsync(&sh, shift, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    DD_CUDA(cudaStreamSynchronize(c->stream));
    out_h->sigma = h.rho;
    out_h->eta = h.eta;
    out_h->drho = h.drho;
    out_h->iters = h.iters;
    out_h->status = h.done ? h.status : DD_EMAXIT;
    out_h->shift = sh;
    DD_CUDA(cudaFreeAsync(Gi, c->stream));
    DD_CUDA(cudaFreeAsync(Gn, c->stream));
    DD_CUDA(cudaFreeAsync(y, c->stream));
    DD_CUDA(cudaFreeAsync(w, c->stream));
    DD_CUDA(cudaFreeAsync(cs, c->stream));
  }
  DD_CUDA(cudaFreeAsync(CB, c->stream));
  DD_CUDA(cudaFreeAsync(RB, c->stream));
  DD_CUDA(cudaFreeAsync(inv, c->stream));
  DD_CUDA(cudaFreeAsync(nvec, c->stream));
  DD_CUDA(cudaStreamSynchronize(c->stream));
  return ok;
}

// Two phases: shift s0 = min V - 1 (safe) until the Rayleigh quotient has settled to 1e-6,
// then s1 = rho - 0.02 (rho - s0), warm-started, to full accuracy.  The refined shift is
// below sigma_1 whenever the eigenvalue error is under 2% of rho - s0; if it is not, the
// factorisation meets a non-positive pivot and the solve continues with the safe shift
// (a larger margin is tried first).
int cell_eigenpair(dd_ctx* c) {
  const Geo& g = c->g;
  const int ncol = (g.p == 1) ? g.n : g.n * g.n;
  c->ncell = (long long)ncol * g.nyi;
  c->cell_band = (g.p == 1) ? 2 * g.nyi + 1 : 2 * g.n * g.nyi + 2 * g.nyi + 1;
  double* shift = nullptr;
  DD_CUDA(cudaMallocAsync(&shift, sizeof(double), c->stream));
  CellOut h{};
  if (!cell_phase(c, shift, true, 0.0, 0, 1e-6, 1e-3, 20000, &h)) {
    DD_CUDA(cudaFreeAsync(shift, c->stream));
    throw Error(DD_ENOTSPD, "cell matrix A_# - s M_# not positive definite");
  }
  if (h.status != 0 && h.status != DD_EMAXIT) throw Error(h.status, "cell inverse iteration failed");
  int iters = h.iters;
  CellOut h1 = h;
  bool refined = false;
  for (double frac : {0.02, 0.2}) {
    CellOut h2 = h1;
    if (cell_phase(c, shift, false, frac, 1, 1e-14, 1e-10, 2000, &h2)) {
      h = h2;
      iters += h2.iters;
      refined = true;
      break;
    }
  }
  if (!refined) {
    if (!cell_phase(c, shift, true, 0.0, 1, 1e-14, 1e-10, 20000, &h)) throw Error(DD_ENOTSPD, "cell factorisation");
    iters += h.iters;
  }
  DD_CUDA(cudaFreeAsync(shift, c->stream));
  DD_CUDA(cudaStreamSynchronize(c->stream));
  if (h.status != 0 && h.status != DD_EMAXIT) throw Error(h.status, "cell inverse iteration failed");
  c->sigma = h.sigma;
  c->cell_iters = iters;
  return h.status;
}

}  // namespace dd
