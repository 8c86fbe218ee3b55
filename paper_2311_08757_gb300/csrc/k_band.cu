// Local subdomain matrices and their banded Cholesky factors; the FP64 local solves of
// the plain method; the cell eigenpair.
//
// Local problems (Sec. 3.1): A_{sigma,i} = R_i A_sigma R_i^T on the interior nodes strictly
// inside the open overlapping box Omega_i (homogeneous Dirichlet on its artificial
// boundary).  All subdomains with the same clipping (left / interior / right per axis) have
// identical matrices, because the cells are translated copies and V is periodic (A1); the
// factors are stored once per type.  Local order: (c1, c2, j) with j fastest, so the
// half bandwidth is nyi + 1 (p = 1) or w2 nyi + nyi + 1 (p = 2).
#include <algorithm>
#include <atomic>

#include "dd_band.cuh"
#include "dd_ritz.cuh"

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

__device__ __forceinline__ double rsqrt_el(double v) { return rsqrt(v); }
__device__ __forceinline__ float rsqrt_el(float v) { return rsqrtf(v); }

// T = double, or float for factors whose inverses are rounded to a tensor-core type and for
// the cell preconditioner (GB300 issues FP32 at 64x the FP64 rate)
template <typename T, int P, int PPT>
__global__ void __launch_bounds__(1024) k_band_factor_win(T* CB, T* inv, const int* __restrict__ nvec,
                                                          int nmax, int b, int* flag) {
  extern __shared__ __align__(16) unsigned char fsm_raw[];
  T* fsm = reinterpret_cast<T*>(fsm_raw);
  const int m = blockIdx.x;
  const int n = nvec[m];
  const int bs = b + 1, W = b + 1;
  // window column stride: even, so that the update's address step between consecutive
  // threads (stride - 1 words per d2) is odd and their shared-memory banks differ (a stride of
  // b + 1 = 33 for b = 32 put a whole warp on one bank)
  const int S = (bs + 1) & ~1;
  const int t = threadIdx.x;   // owns entry d = t of the columns it stages (bs <= blockDim.x)
  T* win = fsm;               // W columns x S entries
  T* colk = fsm + W * S;      // L(k+d, k), d = 0..b
  T* rq = colk + bs;          // P entering columns in flight (cp.async), P x bs
  T* A = CB + (size_t)m * nmax * bs;
  T* iv = inv + (size_t)m * nmax;
  // this thread's pairs (d1, d2), 1 <= d2 <= d1 <= b, of the lower triangle of the window
  // update: linear index e = d1 (d1 - 1) / 2 + d2 - 1 taken as e = t, t + T, ...; in that order
  // d1 never decreases, so the pairs beyond the last column's reach form a suffix
  // exactly PPT pair slots per thread (the block is sized for it), unrolled so that their
  // shared-memory loads issue together; an absent pair is (d1, d2) = (255, 0), beyond reach
  unsigned pr[(PPT + 1) / 2];   // two pairs per word: (d1 << 8 | d2) in each half (b <= 160 < 255)
  {
    const int T = (int)blockDim.x, tot = b * (b + 1) / 2;
#pragma unroll
    for (int j = 0; j < PPT; ++j) {
      const int e = t + j * T;
      int d1 = 255, d2 = 0;
      if (e < tot) {
        d1 = (int)((sqrtf(8.0f * (float)e + 1.0f) + 1.0f) * 0.5f);   // first guess, then exact
        while (d1 * (d1 - 1) / 2 > e) --d1;
        while ((d1 + 1) * d1 / 2 <= e) ++d1;
        d2 = e - d1 * (d1 - 1) / 2 + 1;
      }
      const unsigned half = ((unsigned)d1 << 8) | (unsigned)d2;
      if (j & 1) pr[j >> 1] |= half << 16;
      else pr[j >> 1] = half;
    }
  }
  const int first = min(W, n);
  for (int e = t; e < first * bs; e += blockDim.x) win[(e / bs) * S + e % bs] = A[e];
  // entering columns are copied P steps before they are needed, asynchronously into a
  // shared ring (cp.async: a block barrier waits for a thread's outstanding loads, not for its
  // asynchronous copies), one commit group per step; each thread reads back only what it copied
#pragma unroll
  for (int u = 0; u < P; ++u) {
    if (t < bs) cp_async_el(rq + u * bs + t, A + (size_t)min(W + u, n - 1) * bs + t);
    cp_async_commit();
  }
  __syncthreads();
  int sk = 0;   // ring slot of column k: k mod W, kept incrementally
  for (int k0 = 0; k0 < n; k0 += P) {
#pragma unroll
    for (int u = 0; u < P; ++u) {
      const int k = k0 + u;
      if (k < n) {
        T il;
        if constexpr (sizeof(T) == 4) {
          // FP32: every thread forms the pivot's reciprocal square root itself (identical
          // values), which saves the barrier that publishing it would take
          T piv = win[sk * S];
          if (!(piv > (T)0)) {
            if (t == 0) atomicOr(flag, 1);
            piv = (T)1;
          }
          il = rsqrt_el(piv);
          if (t == 0) {
            A[(size_t)k * bs] = piv * il;
            iv[k] = il * il;
          }
        } else {
          // FP64: one thread (the FP64 pipe would pay for every redundant copy)
          if (t == 0) {
            T piv = win[sk * S];
            if (!(piv > (T)0)) {
              atomicOr(flag, 1);
              piv = (T)1;
            }
            const T l = rsqrt_el(piv);
            A[(size_t)k * bs] = piv * l;
            iv[k] = l * l;
            colk[0] = l;
          }
          __syncthreads();
          il = colk[0];
        }
        const int dmax = min(b, n - 1 - k);
        for (int d = 1 + t; d <= b; d += blockDim.x) {
          T v = (T)0;
          if (d <= dmax) {
            v = win[sk * S + d] * il;            // L(k+d, k)
            A[(size_t)k * bs + d] = v * il;      // pre-scaled by 1/L(k,k)
          }
          colk[d] = v;
        }
        __syncthreads();
        // A(k+d1, k+d2) -= L(k+d1, k) L(k+d2, k) over this thread's pairs with d1 <= dmax;
        // these touch the slots of columns k+1..k+b only
#pragma unroll
        for (int j = 0; j < PPT; ++j) {
          const unsigned half = (j & 1) ? (pr[j >> 1] >> 16) : (pr[j >> 1] & 0xFFFFu);
          const int d1 = (int)(half >> 8), d2 = (int)(half & 0xFFu);
          if (d1 <= dmax) {
            int slot = sk + d2;                  // ring slot of column k + d2
            if (slot >= W) slot -= W;
            T* a = win + slot * S + (d1 - d2);
            *a = fma_el(-colk[d1], colk[d2], *a);
          }
        }
        // the slot of column k is free (read before the barrier above): store column k + W
        // (untouched so far, copied P steps ago) and start the copy of k + W + P
        cp_async_wait<P - 1>();
        if (k + W < n && t < bs) win[sk * S + t] = rq[u * bs + t];
        if (t < bs) cp_async_el(rq + u * bs + t, A + (size_t)min(k + W + P, n - 1) * bs + t);
        cp_async_commit();
        __syncthreads();
        sk = (sk + 1 == W) ? 0 : sk + 1;
      }
    }
  }
  cp_async_wait<0>();   // no copy into this block's shared memory outlives it
}

// Wide bands (b > 160, the window does not fit in shared memory): blocked right-looking band
// Cholesky.  Panels of kPanel columns: one CTA per matrix factors the panel in shared memory
// (its columns have received every earlier update; within the panel the updates are rank 1),
// writes the factor in the band storage the solves expect and the panel's unscaled L to a
// scratch; then the rank-kPanel update of the trailing window, A(i, j) -= sum_c L(i, c) L(j, c)
// for k1 <= j <= i <= k1 - 1 + b, is spread over many CTAs, each holding the panel in shared
// memory.  The host steps through the panels (two launches each; no device-side waits).
// Panel width np <= 32, as many columns as shared memory holds.
constexpr int kPanel = 32;

template <typename T>
__global__ void __launch_bounds__(1024) k_bpanel_factor(T* CB, T* inv, T* Lp, const int* __restrict__ nvec, int nmax,
                                                       int b, int np, int k0, int* flag) {
  extern __shared__ __align__(16) unsigned char bp_raw[];
  T* P = reinterpret_cast<T*>(bp_raw);   // panel columns: P[c * bs + d] = A(k0 + c + d, k0 + c)
  const int m = blockIdx.x, n = nvec[m];
  if (k0 >= n) return;
  const int bs = b + 1, nb = min(np, n - k0);
  T* A = CB + (size_t)m * nmax * bs;
  T* iv = inv + (size_t)m * nmax;
  T* L = Lp + (size_t)m * np * bs;
  for (int e = threadIdx.x; e < nb * bs; e += blockDim.x) P[e] = A[(size_t)k0 * bs + e];
  __syncthreads();
  for (int c = 0; c < nb; ++c) {
    const int k = k0 + c;
    T piv = P[c * bs];
    if (!(piv > (T)0)) {
      if (threadIdx.x == 0) atomicOr(flag, 1);
      piv = (T)1;
    }
    const T il = rsqrt_el(piv);   // every thread
    const int dmax = min(b, n - 1 - k);
    for (int d = threadIdx.x; d <= b; d += blockDim.x) {
      if (d == 0) {   // P[c * bs] stays the pivot: every thread reads it above, none after
        A[(size_t)k * bs] = piv * il;   // L(k, k)
        iv[k] = il * il;
        L[c * bs] = piv * il;
      } else {
        const T l = (d <= dmax) ? P[c * bs + d] * il : (T)0;   // L(k + d, k)
        A[(size_t)k * bs + d] = l * il;   // pre-scaled by 1 / L(k, k) (0 past the end)
        P[c * bs + d] = l;
        L[c * bs + d] = l;
      }
    }
    __syncthreads();
    // the later panel columns c2 > c: A(j + d2, j) -= L(j + d2, k) L(j, k), j = k0 + c2
    const int rem = nb - 1 - c;
    for (int e = threadIdx.x; e < rem * bs; e += blockDim.x) {
      const int c2 = c + 1 + e / bs, d2 = e % bs;
      const int ei = c2 - c + d2;   // row offset from k
      if (ei <= b) P[c2 * bs + d2] = fma_el(-P[c * bs + ei], P[c * bs + (c2 - c)], P[c2 * bs + d2]);
    }
    __syncthreads();
  }
}

// tile (blockIdx.x) of 32 trailing columns of matrix blockIdx.y
template <typename T>
__global__ void __launch_bounds__(1024) k_bpanel_update(T* CB, const T* __restrict__ Lp,
                                                       const int* __restrict__ nvec, int nmax, int b, int np,
                                                       int k0) {
  extern __shared__ __align__(16) unsigned char bu_raw[];
  T* Ls = reinterpret_cast<T*>(bu_raw);   // the panel's L: Ls[c * bs + e] = L(k0 + c + e, k0 + c)
  const int m = blockIdx.y, n = nvec[m];
  const int nb = min(np, n - k0);
  if (nb <= 0) return;
  const int k1 = k0 + nb, last = min(k1 - 1 + b, n - 1);   // rows and columns the panel reaches
  const int j0 = k1 + 32 * blockIdx.x;
  if (j0 > last) return;
  const int bs = b + 1;
  const T* L = Lp + (size_t)m * np * bs;
  for (int e = threadIdx.x; e < nb * bs; e += blockDim.x) Ls[e] = L[e];
  __syncthreads();
  T* A = CB + (size_t)m * nmax * bs;
  const int ncol = min(32, last - j0 + 1);
  for (int e = threadIdx.x; e < ncol * bs; e += blockDim.x) {
    const int jj = e / bs, r = e % bs;   // entry (i, j) = (j + r, j), stored at CB[j][r]
    const int j = j0 + jj, i = j + r;
    if (i > last) continue;
    T acc = (T)0;
#pragma unroll 8
    for (int c = 0; c < nb; ++c) {
      const int ei = i - k0 - c, ej = j - k0 - c;   // ej >= 1; both past the band give 0
      if (ei <= b) acc = fma_el(Ls[c * bs + ei], Ls[c * bs + ej], acc);
    }
    A[(size_t)j * bs + r] -= acc;
  }
}

// launch the factorisation of nmat band matrices (sizes in nvec) and build the row band
template <typename T>
static void factor_launch(T* CB, T* RB, T* inv, const int* nvec, int nmat, int nmax, int b, int* flag,
                          cudaStream_t s);

// RB[i][d] = L(i, i-d) = CB[i-d][d]
template <typename T>
__global__ void k_band_rows(const T* __restrict__ CB, T* RB, const int* __restrict__ nvec,
                            int nmat, int nmax, int b) {
  const int bs = b + 1;
  const long long total = (long long)nmat * nmax * bs;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const int m = (int)(t / ((long long)nmax * bs));
    const long long rem = t - (long long)m * nmax * bs;
    const int i = (int)(rem / bs), d = (int)(rem % bs);
    const int n = nvec[m];
    T v = (T)0;
    if (i < n && i - d >= 0) v = CB[((size_t)m * nmax + (i - d)) * bs + d];
    RB[t] = v;
  }
}

template <typename T>
int launch_band_factor(dd_ctx* c, T* CB, T* RB, T* inv, int nmat, int nmax, int b, int* flag,
                       const int* sizes_host) {
  int* nvec = nullptr;
  DD_CUDA(cudaMallocAsync(&nvec, sizeof(int) * nmat, c->stream));
  std::vector<int> nh(nmat, nmax);
  if (sizes_host != nullptr)
    for (int t = 0; t < nmat; ++t) nh[t] = sizes_host[t];
  DD_CUDA(cudaMemcpyAsync(nvec, nh.data(), sizeof(int) * nmat, cudaMemcpyHostToDevice, c->stream));
  factor_launch(CB, RB, inv, nvec, nmat, nmax, b, flag, c->stream);
  DD_CUDA(cudaFreeAsync(nvec, c->stream));
  return DD_OK;
}
template int launch_band_factor<double>(dd_ctx*, double*, double*, double*, int, int, int, int*, const int*);
template int launch_band_factor<float>(dd_ctx*, float*, float*, float*, int, int, int, int*, const int*);

template <typename T>
static void factor_launch(T* CB, T* RB, T* inv, const int* nvec, int nmat, int nmax, int b, int* flag,
                          cudaStream_t s) {
  if (b <= kBandWinMax) {
    const size_t smem = sizeof(T) * ((size_t)(b + 1) * (((b + 1) + 1) & ~1) + (size_t)(b + 1) * (1 + 4));
    // PPT triangle pairs per thread, the block at least one thread per entry of a column (the
    // window's entering columns are staged one entry per thread) and at most 1024 threads
    const int tot = b * (b + 1) / 2;
    // four pairs per thread where the block stays within 1024 threads (measured at b = 63:
    // 4 pairs x 16 warps 0.53 ms, 16 pairs x 4 warps 0.90 ms: the wider block hides latency)
    const int ppt = tot <= 2048 ? 4 : (tot <= 4096 ? 8 : 16);
    int threads = ((tot + ppt - 1) / ppt + 31) / 32 * 32;
    threads = std::max(threads, (b + 1 + 31) / 32 * 32);
    threads = std::min(threads, 1024);
#define DD_FWIN(PPT_)                                                                                         \
  do {                                                                                                      \
    static dd::PerDeviceOnce attr;   /* once per device and instance */                                     \
    dd::once_per_device(attr, [] {                                                                          \
      DD_CUDA(cudaFuncSetAttribute(k_band_factor_win<T, 4, PPT_>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                                   220 * 1024));                                                            \
    });                                                                                                     \
    (k_band_factor_win<T, 4, PPT_><<<nmat, threads, smem, s>>>(CB, inv, nvec, nmax, b, flag), dd::note_launch()); \
  } while (0)
    if (ppt == 4) DD_FWIN(4);
    else if (ppt == 8) DD_FWIN(8);
    else DD_FWIN(16);
#undef DD_FWIN
  } else {
    const int np = std::min<int>(kPanel, (int)((200 * 1024) / (sizeof(T) * (size_t)(b + 1))));
    if (np < 1) throw Error(DD_EINVAL, "band too wide for the shared-memory panel factorisation");
    T* Lp = nullptr;
    DD_CUDA(cudaMallocAsync(&Lp, sizeof(T) * (size_t)nmat * np * (b + 1), s));
    const size_t psm = sizeof(T) * (size_t)np * (b + 1);
    static PerDeviceOnce attr;   // once per device and type
    once_per_device(attr, [] {
      DD_CUDA(cudaFuncSetAttribute(k_bpanel_factor<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024));
      DD_CUDA(cudaFuncSetAttribute(k_bpanel_update<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024));
    });
    const dim3 ug((b + 31) / 32, nmat);
    for (int k0 = 0; k0 < nmax; k0 += np) {
      (k_bpanel_factor<T><<<nmat, 1024, psm, s>>>(CB, inv, Lp, nvec, nmax, b, np, k0, flag), dd::note_launch());
      (k_bpanel_update<T><<<ug, 1024, psm, s>>>(CB, Lp, nvec, nmax, b, np, k0), dd::note_launch());
    }
    DD_CUDA(cudaFreeAsync(Lp, s));
  }
  DD_CUDA(cudaGetLastError());
  const long long total = (long long)nmat * nmax * (b + 1);
  (k_band_rows<T><<<grid_blocks(total, kThreads), kThreads, 0, s>>>(CB, RB, nvec, nmat, nmax, b), dd::note_launch());
  DD_CUDA(cudaGetLastError());
}

// ----------------------------------------------------------------------------------------
// Local matrix assembly from the A_sigma stencil table: CB[t][k][k'-k] = A_sigma(k', k), k' >= k.
// ----------------------------------------------------------------------------------------
template <typename T>
__global__ void k_local_assemble(Geo g, const double* __restrict__ tabS, const Sub* __restrict__ rep,
                                 int ntypes, int nmax, int b, T* CB) {
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
    T* row = CB + ((size_t)ty * nmax + k) * bs;
    for (int tap = 0; tap < g.ntap; ++tap) {
      int d1, d2 = 0, dy;
      if (g.p == 1) { d1 = tap / 3 - 1; dy = tap % 3 - 1; }
      else { d1 = tap / 9 - 1; d2 = (tap / 3) % 3 - 1; dy = tap % 3 - 1; }
      const int n1 = c1 + d1, n2 = c2 + d2, nj = sj + dy;
      if (n1 < 0 || n1 >= s.w1 || n2 < 0 || n2 >= s.w2 || nj < 0 || nj >= g.nyi) continue;
      const int kk = (n1 * s.w2 + n2) * g.nyi + nj;
      if (kk < k) continue;
      row[kk - k] = (T)tabS[(size_t)tap * g.ncls + cls];
    }
  }
}

template <typename T>
void launch_local_assemble(dd_ctx* c, T* CB) {
  // representative subdomain of every type
  std::vector<Sub> rep(c->ntypes);
  for (int t = 0; t < c->ntypes; ++t) {
    for (const Sub& s : c->subs_h)
      if (s.type == t) { rep[t] = s; break; }
  }
  Sub* drep = nullptr;
  DD_CUDA(cudaMallocAsync(&drep, sizeof(Sub) * c->ntypes, c->stream));
  DD_CUDA(cudaMemcpyAsync(drep, rep.data(), sizeof(Sub) * c->ntypes, cudaMemcpyHostToDevice, c->stream));
  const size_t nbytes = sizeof(T) * (size_t)c->ntypes * c->nloc_max * (c->band + 1);
  DD_CUDA(cudaMemsetAsync(CB, 0, nbytes, c->stream));
  const long long total = (long long)c->ntypes * c->nloc_max;
  (k_local_assemble<T><<<grid_blocks(total, 128), 128, 0, c->stream>>>(c->g, c->tabS, drep, c->ntypes,
                                                                      c->nloc_max, c->band, CB), dd::note_launch());
  DD_CUDA(cudaGetLastError());
  DD_CUDA(cudaFreeAsync(drep, c->stream));
}
template void launch_local_assemble<double>(dd_ctx*, double*);
template void launch_local_assemble<float>(dd_ctx*, float*);

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
  constexpr int RING = band_ring_elems<NV, PF>();
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
        if (c0 != nullptr) cr = fma(wt[loc_pad(g, k)], v, cr);
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
    for (int k = lane; k < n; k += 32) y[loc_pad(g, k)] = xs[(size_t)j * nmax + k];
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
      static PerDeviceOnce attr_set;   // once per device and instance
      once_per_device(attr_set, [] {
        DD_CUDA(cudaFuncSetAttribute(k_local_solve<NV, PF, KK>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     220 * 1024));
      });
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
// A_# psi = sigma M_# psi with x-periodic, y-Dirichlet conditions.  The factor of the shifted
// cell matrix uses an interleaved x order (0, n-1, 1, n-2, ...) that keeps periodic
// neighbours within two positions, so the periodic operator is banded.
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
template <typename T>
__global__ void k_cell_assemble(Geo g, const double* __restrict__ tabA, const double* __restrict__ tabM,
                                const double* __restrict__ shift, int b, T* CB) {
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
      CB[(size_t)row * bs + (col - row)] += (T)(tabA[ti] - s * tabM[ti]);
    }
  }
}

// value at natural cell index k of the periodic cell stencil T x; the taps are unrolled so
// that all their loads are in flight at once (x-periodic wrap by compare and add)
template <int P>
__device__ __forceinline__ double cell_at(const Geo& g, const double* __restrict__ tab, const double* __restrict__ x,
                                          int k) {
  const int sj = k % g.nyi, cc = k / g.nyi;
  const int a1 = (P == 1) ? cc : cc / g.n, a2 = (P == 1) ? 0 : cc % g.n;
  const int cls = ((P == 1) ? a1 : a1 * g.n + a2) * g.Ypad + sj;
  double acc = 0.0;
#pragma unroll
  for (int tap = 0; tap < (P == 1 ? 9 : 27); ++tap) {
    const int d1 = (P == 1) ? tap / 3 - 1 : tap / 9 - 1;
    const int d2 = (P == 1) ? 0 : (tap / 3) % 3 - 1;
    const int dy = tap % 3 - 1;
    const int nj = sj + dy;
    int b1 = a1 + d1;
    b1 += (b1 < 0) ? g.n : 0;
    b1 -= (b1 >= g.n) ? g.n : 0;
    int b2 = a2 + d2;
    if (P == 2) {
      b2 += (b2 < 0) ? g.n : 0;
      b2 -= (b2 >= g.n) ? g.n : 0;
    }
    const bool ok = nj >= 0 && nj < g.nyi;
    const int kk = ((P == 1) ? b1 : b1 * g.n + b2) * g.nyi + (ok ? nj : sj);   // in range either way
    const double tv = __ldg(tab + (size_t)tap * g.ncls + cls), xv = x[kk];
    if (ok) acc = fma(tv, xv, acc);
  }
  return acc;
}

// ---- cell eigen-solve: LOPCG preconditioned by an FP32 shift-and-invert ------------------
// The lowest eigenpair of A_# psi = sigma M_# psi by locally optimal preconditioned
// iterations on S = [x_k, w_k, x_{k-1}] with w_k = T (A_# x_k - rho_k M_# x_k) (the same
// Rayleigh-Ritz step as Algorithm 1), where T is the dense inverse of A_# - s M_#,
// s = min V - 1 (SPD because M_V >= min(V) M for a quadrature with positive weights), formed
// in FP32 from an FP32 banded Cholesky.  T only steers the search direction: every residual,
// Gram matrix and Rayleigh quotient is formed in FP64 from the FP64 stencils, so the pair is
// accurate to FP64 whatever T's rounding.  One factorisation and one inverse replace the
// two FP64 factorisations of a two-shift inverse iteration; the FP32 factor runs at GB300's
// FP32 rate (64 lanes per FP64 lane).
struct CellLop {
  LopState ls;   // Gram matrices, Ritz coefficients and value (theta) of the last step
  double rho, rho_prev, eta, eta_prev, drho, xmx;
  int iters, stable, done, status;
};

constexpr int kCellBlock = 64;   // small blocks: the cell vectors are short, spread them over SMs

template <typename T>
__global__ void k_cell_perm_dense(Geo g, int ncell, const T* __restrict__ Gi, T* __restrict__ Gn) {
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

// theta_0 = x^T A_# x / x^T M_# x of the start vector
template <int P>
__global__ void __launch_bounds__(kCellBlock) k_cl_init(Geo g, int ncell, const double* __restrict__ tabA,
                                                        const double* __restrict__ tabM, const double* __restrict__ x,
                                                        CellLop* cl, double* partials, unsigned* counter) {
  double acc[2] = {0.0, 0.0};
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < ncell; k += gridDim.x * blockDim.x) {
    acc[0] = fma(x[k], cell_at<P>(g, tabA, x, k), acc[0]);
    acc[1] = fma(x[k], cell_at<P>(g, tabM, x, k), acc[1]);
  }
  double tot[2];
  if (grid_sum_last<2>(acc, partials, counter, tot) && threadIdx.x == 0) {
    cl->ls.theta = tot[0] / tot[1];
    if (!(tot[1] > 0.0) || !isfinite(cl->ls.theta)) {
      cl->status = DD_ENAN;
      cl->done = 1;
    }
  }
}

// r = A_# x - theta M_# x (to FP32 for the preconditioner), rho = Rayleigh quotient of x,
// eta = ||A x - rho M x|| / (|rho| ||M x||) (with theta, the Ritz value, equal to rho up to
// rounding), and the stop rule
template <int P>
__global__ void __launch_bounds__(kCellBlock) k_cl_resid(Geo g, int ncell, const double* __restrict__ tabA,
                                                         const double* __restrict__ tabM, const double* __restrict__ x,
                                                         float* __restrict__ rf, double tol_eta,
                                                         int maxit, CellLop* cl, double* partials, unsigned* counter) {
  if (cl->done) return;
  const double th = cl->ls.theta;
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < ncell; k += gridDim.x * blockDim.x) {
    const double ax = cell_at<P>(g, tabA, x, k), mx = cell_at<P>(g, tabM, x, k);
    const double r = fma(-th, mx, ax);
    rf[k] = __double2float_rn(r);
    acc[0] = fma(r, r, acc[0]);
    acc[1] = fma(mx, mx, acc[1]);
    acc[2] = fma(x[k], ax, acc[2]);
    acc[3] = fma(x[k], mx, acc[3]);
  }
  double tot[4];
  if (grid_sum_last<4>(acc, partials, counter, tot) && threadIdx.x == 0) {
    const double rho = tot[2] / tot[3];
    const double eta = sqrt(tot[0] / tot[1]) / fabs(rho);
    const double drho = fabs(rho - cl->rho_prev);
    cl->iters += 1;
    cl->rho = rho;
    cl->eta = eta;
    cl->drho = drho;
    cl->xmx = tot[3];
    if (!isfinite(rho) || !isfinite(eta)) {
      cl->status = DD_ENAN;
      cl->done = 1;
    } else {
      // past the residual target, go on while the residual still halves: psi enters the
      // coarse space twice (A_0 = Z^T A_sigma Z), so it is driven to its rounding floor, which
      // the cheap steps reach a few steps later (the Rayleigh quotient, error ~ eta^2, has long
      // been stationary by then).  Near the floor the residual alternates between halving and
      // not, so every non-halving step below the target counts, and a residual 1e-3 below the
      // target counts at once.
      if (eta <= tol_eta) {
        if (eta >= 0.5 * cl->eta_prev || eta <= 1e-3 * tol_eta) cl->stable += 1;
      } else {
        cl->stable = 0;
      }
      if (cl->stable >= 2) cl->done = 1;
      else if (cl->iters >= maxit) {
        cl->status = DD_EMAXIT;
        cl->done = 1;
      }
    }
    cl->eta_prev = eta;
    cl->rho_prev = rho;
  }
}

// w = T r, warp per row, FP32 (T steers the search direction only)
__global__ void k_cl_gemv(int n, const float* __restrict__ G, const float* __restrict__ r, double* __restrict__ w,
                          const CellLop* cl) {
  if (cl->done) return;
  const int lane = threadIdx.x & 31;
  const int row = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (row >= n) return;
  const float* gr = G + (size_t)row * n;
  float acc = 0.0f;
  for (int k = lane; k < n; k += 32) acc = fmaf(__ldg(gr + k), __ldg(r + k), acc);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(kFull, acc, o);
  if (lane == 0) w[row] = f32_to_f64(acc);
}

// Gram matrices of S = [x, w, xp] under A_# and M_# (images formed on the fly: the cell
// vectors are short) and the Rayleigh-Ritz step in the last block
template <int P>
__global__ void __launch_bounds__(kCellBlock) k_cl_gram(Geo g, int ncell, const double* __restrict__ tabA,
                                                        const double* __restrict__ tabM, const double* __restrict__ x,
                                                        const double* __restrict__ w, const double* __restrict__ xp,
                                                        CellLop* cl, double* partials, unsigned* counter,
                                                        double drop) {
  if (cl->done) return;
  double acc[15];
#pragma unroll
  for (int k = 0; k < 15; ++k) acc[k] = 0.0;
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < ncell; k += gridDim.x * blockDim.x) {
    const double v[3] = {x[k], w[k], xp[k]};
    const double a[3] = {cell_at<P>(g, tabA, x, k), cell_at<P>(g, tabA, w, k), cell_at<P>(g, tabA, xp, k)};
    const double m[3] = {cell_at<P>(g, tabM, x, k), cell_at<P>(g, tabM, w, k), cell_at<P>(g, tabM, xp, k)};
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = i; j < 3; ++j) {
        acc[sym3(i, j)] = fma(v[i], a[j], acc[sym3(i, j)]);
        acc[6 + sym3(i, j)] = fma(v[i], m[j], acc[6 + sym3(i, j)]);
      }
#pragma unroll
    for (int i = 0; i < 3; ++i) acc[12 + i] += v[i];
  }
  double tot[15];
  if (grid_sum_last<15>(acc, partials, counter, tot) && threadIdx.x == 0) {
    LopState* ls = &cl->ls;
    for (int k = 0; k < 6; ++k) {
      ls->GA[k] = tot[k];
      ls->GB[k] = tot[6 + k];
    }
    for (int k = 0; k < 3; ++k) ls->sums[k] = tot[12 + k];
    ls->status = 0;
    rayleigh_ritz3(ls, drop);
    if (ls->status != 0) {
      cl->status = ls->status;
      cl->done = 1;
    }
  }
}

// x_{k+1} = c0 x_k + c1 w_k + c2 x_{k-1}
__global__ void k_cl_update(int ncell, const double* __restrict__ x, const double* __restrict__ w,
                            const double* __restrict__ xp, double* __restrict__ xn, const CellLop* cl) {
  if (cl->done) return;
  const double c0 = cl->ls.c[0], c1 = cl->ls.c[1], c2 = cl->ls.c[2];
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < ncell; k += gridDim.x * blockDim.x)
    xn[k] = fma(c0, x[k], fma(c1, w[k], c2 * xp[k]));
}

// psi = x / ||x||_M
__global__ void k_cl_final(int ncell, const double* __restrict__ x, double* __restrict__ psi, const CellLop* cl) {
  const double sc = 1.0 / sqrt(cl->xmx);
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < ncell; k += gridDim.x * blockDim.x) psi[k] = sc * x[k];
}

int cell_eigenpair(dd_ctx* c) {
  const Geo& g = c->g;
  const int ncol = (g.p == 1) ? g.n : g.n * g.n;
  const int ncell = ncol * g.nyi;
  c->ncell = ncell;
  const int b = (g.p == 1) ? 2 * g.nyi + 1 : 2 * g.n * g.nyi + 2 * g.nyi + 1;
  c->cell_band = b;
  cudaStream_t s = c->stream;
  // ---- T = (A_# - s M_#)^{-1} in FP32, natural cell order
  const size_t cbsz = sizeof(float) * (size_t)ncell * (b + 1);
  const size_t gsz = sizeof(float) * (size_t)ncell * ncell;
  float *CB = nullptr, *RB = nullptr, *inv = nullptr, *Gi = nullptr, *Gn = nullptr, *rf = nullptr;
  double *shift = nullptr, *vec = nullptr, *part = nullptr;
  CellLop* cl = nullptr;
  int* flag = c->dev_err + 1;
  DD_CUDA(cudaMallocAsync(&shift, sizeof(double), s));
  DD_CUDA(cudaMallocAsync(&CB, cbsz, s));
  DD_CUDA(cudaMallocAsync(&RB, cbsz, s));
  DD_CUDA(cudaMallocAsync(&inv, sizeof(float) * ncell, s));
  DD_CUDA(cudaMallocAsync(&Gi, gsz, s));
  DD_CUDA(cudaMallocAsync(&Gn, gsz, s));
  DD_CUDA(cudaMallocAsync(&rf, sizeof(float) * ncell, s));
  DD_CUDA(cudaMallocAsync(&vec, sizeof(double) * 4 * (size_t)ncell, s));   // three iterates and w
  DD_CUDA(cudaMallocAsync(&cl, sizeof(CellLop), s));
  DD_CUDA(cudaMallocAsync(&part, sizeof(double) * 15 * kMaxRedBlocks, s));   // block partials of the sums
  DD_CUDA(cudaMemsetAsync(CB, 0, cbsz, s));
  DD_CUDA(cudaMemsetAsync(flag, 0, sizeof(int), s));
  {
    long long nV = (long long)((g.p == 1) ? g.n : g.n * g.n) * g.ny;
    for (int k = 0; k <= g.p; ++k) nV *= g.Q;
    (k_cell_shift<<<1, 1024, 0, s>>>(c->Vqp, nV, shift), dd::note_launch());
  }
  (k_cell_assemble<float><<<grid_blocks(ncell, 128), 128, 0, s>>>(g, c->tabA, c->tabM, shift, b, CB),
   dd::note_launch());
  launch_band_factor(c, CB, RB, inv, 1, ncell, b, flag, nullptr);
  launch_band_inverse_rows(ncell, b, CB, RB, inv, Gi, s);
  (k_cell_perm_dense<float><<<grid_blocks((long long)ncell * ncell, kThreads), kThreads, 0, s>>>(g, ncell, Gi, Gn),
   dd::note_launch());
  DD_CUDA(cudaGetLastError());
  // ---- LOPCG from x_0 = 1
  double* bufs[3] = {vec, vec + ncell, vec + 2 * (size_t)ncell};
  double* w = vec + 3 * (size_t)ncell;
  {
    std::vector<double> ones((size_t)ncell, 1.0);
    DD_CUDA(cudaMemcpyAsync(bufs[0], ones.data(), sizeof(double) * ncell, cudaMemcpyHostToDevice, s));
    DD_CUDA(cudaMemsetAsync(bufs[2], 0, sizeof(double) * ncell, s));   // x_{-1} = 0: dropped by the first step
    CellLop init{};
    init.rho_prev = 1e300;
    init.eta_prev = 1e300;
    DD_CUDA(cudaMemcpyAsync(cl, &init, sizeof(init), cudaMemcpyHostToDevice, s));
    DD_CUDA(cudaStreamSynchronize(s));   // the host vectors above are temporaries
  }
  const int nbv = std::min((ncell + kCellBlock - 1) / kCellBlock, 152 * 4);
  const int gemv_blocks = (ncell + 7) / 8;
  unsigned* cnt = c->cnt + CNT_CELL;
  const int maxit = 400;
  const double drop = 1e-10;
  const bool p1 = g.p == 1;
  if (p1) (k_cl_init<1><<<nbv, kCellBlock, 0, s>>>(g, ncell, c->tabA, c->tabM, bufs[0], cl, part, cnt), dd::note_launch());
  else (k_cl_init<2><<<nbv, kCellBlock, 0, s>>>(g, ncell, c->tabA, c->tabM, bufs[0], cl, part, cnt), dd::note_launch());
  CellLop h{};
  for (int it = 0; it < maxit; it += 4) {
    for (int k = 0; k < 4; ++k) {
      const int j = it + k;
      double *x = bufs[j % 3], *xn = bufs[(j + 1) % 3], *xp = bufs[(j + 2) % 3];
      if (p1)
        (k_cl_resid<1><<<nbv, kCellBlock, 0, s>>>(g, ncell, c->tabA, c->tabM, x, rf, 1e-10, maxit, cl, part, cnt),
         dd::note_launch());
      else
        (k_cl_resid<2><<<nbv, kCellBlock, 0, s>>>(g, ncell, c->tabA, c->tabM, x, rf, 1e-10, maxit, cl, part, cnt),
         dd::note_launch());
      (k_cl_gemv<<<gemv_blocks, 256, 0, s>>>(ncell, Gn, rf, w, cl), dd::note_launch());
      if (p1)
        (k_cl_gram<1><<<nbv, kCellBlock, 0, s>>>(g, ncell, c->tabA, c->tabM, x, w, xp, cl, part, cnt, drop),
         dd::note_launch());
      else
        (k_cl_gram<2><<<nbv, kCellBlock, 0, s>>>(g, ncell, c->tabA, c->tabM, x, w, xp, cl, part, cnt, drop),
         dd::note_launch());
      (k_cl_update<<<nbv, kCellBlock, 0, s>>>(ncell, x, w, xp, xn, cl), dd::note_launch());
    }
    DD_CUDA(cudaGetLastError());
    DD_CUDA(cudaMemcpyAsync(&h, cl, sizeof(CellLop), cudaMemcpyDeviceToHost, s));
    DD_CUDA(cudaStreamSynchronize(s));
    if (h.done) break;
  }
  int fl = 0;
  DD_CUDA(cudaMemcpyAsync(&fl, flag, sizeof(int), cudaMemcpyDeviceToHost, s));
  DD_CUDA(cudaStreamSynchronize(s));
  int status = h.done ? h.status : DD_EMAXIT;
  if (h.iters >= 1 && (status == DD_OK || status == DD_EMAXIT)) {
    // the iterate whose residual passed the test: x_j of the step j = iters - 1
    (k_cl_final<<<nbv, kCellBlock, 0, s>>>(ncell, bufs[(h.iters - 1) % 3], c->psi_cell, cl), dd::note_launch());
    DD_CUDA(cudaGetLastError());
  }
  for (void* p : {(void*)shift, (void*)CB, (void*)RB, (void*)inv, (void*)Gi, (void*)Gn, (void*)rf, (void*)vec,
                  (void*)cl, (void*)part})
    DD_CUDA(cudaFreeAsync(p, s));
  DD_CUDA(cudaStreamSynchronize(s));
  if (fl) throw Error(DD_ENOTSPD, "cell matrix A_# - s M_# not positive definite");
  if (status != DD_OK && status != DD_EMAXIT) throw Error(status, "cell eigen-solve failed");
  c->sigma = h.rho;
  c->cell_iters = h.iters;
  return status;
}

}  // namespace dd
