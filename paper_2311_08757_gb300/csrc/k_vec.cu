// Stencil tables, the matrix-free Q1 operator, and the PCG vector kernels.
//
// A = K + M_V and M of the Q1 discretisation (Sec. 2, discrete weak form) are stored as
// periodic stencil tables: because the box mesh is made of translated copies of the cell
// mesh (Sec. 2) and V is 1-periodic in x (assumption A1), the row of node (a, j) depends
// only on (a mod n, j).  tab[tap][cls] holds the coupling of class cls to its neighbour at
// offset tap in {-1,0,1}^d; A_sigma = A - sigma M (Sec. 1.1) is a third table.
#include <algorithm>
#include <atomic>
#include <map>
#include <mutex>

#include "dd_common.cuh"

namespace dd {

__constant__ double c_gpt[kMaxQ];
__constant__ double c_gwt[kMaxQ];

int grid_blocks(long long work, int threads, int max_per_sm) {
  long long b = (work + threads - 1) / threads;
  long long cap = 152LL * max_per_sm;
  if (b > cap) b = cap;
  if (b > kMaxRedBlocks) b = kMaxRedBlocks;
  if (b < 1) b = 1;
  return (int)b;
}

// Grid of a grid-stride kernel capped at the blocks the SMs keep resident at once (from the
// kernel's registers and shared memory, queried once per kernel), so that it runs as one
// wave: a second, partial wave of blocks leaves most SMs idle at its end.
template <typename K>
static int resident_grid(K* kernel, long long work, int threads) {
  static std::mutex mu;
  static std::map<const void*, int> per_sm;
  int occ = 0;
  {
    std::lock_guard<std::mutex> lk(mu);
    auto it = per_sm.find((const void*)kernel);
    if (it != per_sm.end()) occ = it->second;
  }
  if (occ == 0) {
    DD_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kernel, threads, 0));
    occ = std::max(1, std::min(occ, 8));
    std::lock_guard<std::mutex> lk(mu);
    per_sm[(const void*)kernel] = occ;
  }
  return grid_blocks(work, threads, occ);
}

// ----------------------------------------------------------------------------------------
// S4: stencil tables from V at the cell's Gauss points.
// Element (ex, ey) with local node (bx, by) in {0,1}^d; Q1 basis N_b(xi) = prod N1_{b_k}(xi_k),
// N1_0 = 1 - t, N1_1 = t.  Exact element matrices K^e = sum_k (x)_{ax} (ax == k ? K1 : M1),
// M^e = (x) M1 with K1 = [[1,-1],[-1,1]]/h, M1 = [[2,1],[1,2]] h/6, and
// M_V^e[a,b] = h^d sum_q W_q V_q N_a(xi_q) N_b(xi_q).
// ----------------------------------------------------------------------------------------
template <int P>
__global__ void k_build_tables(Geo g, const double* __restrict__ V, double* tabA, double* tabM) {
  constexpr int D = P + 1;
  const long long total = (long long)g.ncls * g.ntap;
  const double h = g.h;
  const int Q = g.Q;
  int nq = 1;
  for (int k = 0; k < D; ++k) nq *= Q;
  double hd = 1.0;
  for (int k = 0; k < D; ++k) hd *= h;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const int tap = (int)(t / g.ncls);
    const int cls = (int)(t - (long long)tap * g.ncls);
    const int slot = cls % g.Ypad;
    const int cx = cls / g.Ypad;
    if (slot >= g.nyi) {
      tabA[t] = 0.0;
      tabM[t] = 0.0;
      continue;
    }
    const int j = slot + 1;
    int c[2], dxs[2], dy;
    if (P == 1) {
      c[0] = cx;
      dxs[0] = tap / 3 - 1;
      dy = tap % 3 - 1;
    } else {
      c[0] = cx / g.n;
      c[1] = cx % g.n;
      dxs[0] = tap / 9 - 1;
      dxs[1] = (tap / 3) % 3 - 1;
      dy = tap % 3 - 1;
    }
    double sA = 0.0, sM = 0.0;
    // elements around the node: local position l per axis (node = element origin + l)
    for (int mask = 0; mask < (1 << D); ++mask) {
      int la[3], lb[3];
      bool ok = true;
      for (int k = 0; k < P; ++k) {
        la[k] = (mask >> (D - 1 - k)) & 1;
        lb[k] = la[k] + dxs[k];
        if (lb[k] < 0 || lb[k] > 1) ok = false;
      }
      la[P] = mask & 1;
      lb[P] = la[P] + dy;
      if (lb[P] < 0 || lb[P] > 1) ok = false;
      if (!ok) continue;
      const int ey = j - la[P];   // 0 <= ey <= ny-1
      int e = 0;
      for (int k = 0; k < P; ++k) {
        int ex = c[k] - la[k];
        ex = (ex % g.n + g.n) % g.n;
        e = e * g.n + ex;
      }
      e = e * g.ny + ey;
      // K^e and M^e
      double me = 1.0, ke = 0.0;
      for (int ax = 0; ax < D; ++ax) me *= (la[ax] == lb[ax] ? 2.0 : 1.0) * h / 6.0;
      for (int kk = 0; kk < D; ++kk) {
        double t2 = 1.0;
        for (int ax = 0; ax < D; ++ax) {
          if (ax == kk) t2 *= (la[ax] == lb[ax] ? 1.0 : -1.0) / h;
          else t2 *= (la[ax] == lb[ax] ? 2.0 : 1.0) * h / 6.0;
        }
        ke += t2;
      }
      // M_V^e
      double mv = 0.0;
      for (int iq = 0; iq < nq; ++iq) {
        int rem = iq;
        double wq = 1.0, na = 1.0, nb = 1.0;
        for (int ax = D - 1; ax >= 0; --ax) {
          const int qa = rem % Q;
          rem /= Q;
          const double xi = c_gpt[qa];
          wq *= c_gwt[qa];
          na *= la[ax] ? xi : 1.0 - xi;
          nb *= lb[ax] ? xi : 1.0 - xi;
        }
        mv = fma(wq * V[(size_t)e * nq + iq], na * nb, mv);
      }
      sA += ke + hd * mv;
      sM += me;
    }
    tabA[t] = sA;
    tabM[t] = sM;
  }
}

void launch_build_tables(dd_ctx* c) {
  const Geo& g = c->g;
  // Gauss-Legendre points and weights on [0, 1] (closed forms).
  double pt[kMaxQ] = {0}, wt[kMaxQ] = {0};
  const int Q = g.Q;
  if (Q == 1) {
    pt[0] = 0.5; wt[0] = 1.0;
  } else if (Q == 2) {
    const double s = 0.5 / sqrt(3.0);
    pt[0] = 0.5 - s; pt[1] = 0.5 + s; wt[0] = wt[1] = 0.5;
  } else if (Q == 3) {
    const double s = 0.5 * sqrt(0.6);
    pt[0] = 0.5 - s; pt[1] = 0.5; pt[2] = 0.5 + s;
    wt[0] = wt[2] = 5.0 / 18.0; wt[1] = 8.0 / 18.0;
  } else {
    const double a = sqrt(3.0 / 7.0 - 2.0 / 7.0 * sqrt(6.0 / 5.0));
    const double b = sqrt(3.0 / 7.0 + 2.0 / 7.0 * sqrt(6.0 / 5.0));
    const double wa = (18.0 + sqrt(30.0)) / 36.0, wb = (18.0 - sqrt(30.0)) / 36.0;
    pt[0] = 0.5 - 0.5 * b; pt[1] = 0.5 - 0.5 * a; pt[2] = 0.5 + 0.5 * a; pt[3] = 0.5 + 0.5 * b;
    wt[0] = wt[3] = 0.5 * wb; wt[1] = wt[2] = 0.5 * wa;
  }
  DD_CUDA(cudaMemcpyToSymbolAsync(c_gpt, pt, sizeof(pt), 0, cudaMemcpyHostToDevice, c->stream));
  DD_CUDA(cudaMemcpyToSymbolAsync(c_gwt, wt, sizeof(wt), 0, cudaMemcpyHostToDevice, c->stream));
  const long long total = (long long)g.ncls * g.ntap;
  const int nb = grid_blocks(total, kThreads);
  if (g.p == 1) (k_build_tables<1><<<nb, kThreads, 0, c->stream>>>(g, c->Vqp, c->tabA, c->tabM), dd::note_launch());
  else (k_build_tables<2><<<nb, kThreads, 0, c->stream>>>(g, c->Vqp, c->tabA, c->tabM), dd::note_launch());
  DD_CUDA(cudaGetLastError());
}

__global__ void k_tabS(long long n, const double* __restrict__ A, const double* __restrict__ M, double sigma,
                       double* S) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n;
       t += (long long)gridDim.x * blockDim.x)
    S[t] = A[t] - sigma * M[t];
}

// S2[cls][tap] = split(S[tap][cls]) for the ntap taps of a class, zero pads up to the stride
__global__ void k_tab_split(int ncls, int ntap, int stride, const double* __restrict__ S, float2* __restrict__ S2) {
  const long long n = (long long)ncls * stride;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n;
       t += (long long)gridDim.x * blockDim.x) {
    const int cls = (int)(t / stride), tap = (int)(t % stride);
    S2[t] = tap < ntap ? f64_split(S[(size_t)tap * ncls + cls]) : make_float2(0.0f, 0.0f);
  }
}

void launch_tabS(dd_ctx* c, double sigma) {
  const long long n = (long long)c->g.ncls * c->g.ntap;
  (k_tabS<<<grid_blocks(n, kThreads), kThreads, 0, c->stream>>>(n, c->tabA, c->tabM, sigma, c->tabS), dd::note_launch());
  DD_CUDA(cudaGetLastError());
  if (c->tabS2) {
    const int stride = pair_tap_stride(c->g.p);
    const long long n2 = (long long)c->g.ncls * stride;
    (k_tab_split<<<grid_blocks(n2, kThreads), kThreads, 0, c->stream>>>(c->g.ncls, c->g.ntap, stride, c->tabS,
                                                                          c->tabS2),
     dd::note_launch());
    DD_CUDA(cudaGetLastError());
  }
}

// ----------------------------------------------------------------------------------------
// K1: matrix-free operator y = T x (T = A_sigma, A or M) over the interior columns.
// ----------------------------------------------------------------------------------------
template <int P, bool DOT>
__device__ __forceinline__ void stencil_body(VBlk vb, Geo g, const double* __restrict__ tab,
                                                      const double* __restrict__ x, double* __restrict__ y,
                                                      double* partials, unsigned* counter, double* out) {
  const long long total = (long long)g.nxi * (P == 2 ? g.nxi : 1) * g.Ypad;
  double acc[1] = {0.0};
  for (long long t = (long long)vb.b * blockDim.x + threadIdx.x; t < total;
       t += (long long)vb.nb * blockDim.x) {
    Node nd = node_of<P>(g, t);
    const int cls = cls_of<P>(g, nd);
    const double v = stencil_at<P>(g, tab, x, nd.idx, cls);
    y[nd.idx] = v;
    if (DOT) acc[0] = fma(x[nd.idx], v, acc[0]);
  }
  if (DOT) {
    double tot[1];
    if (grid_sum_last<1>(acc, partials, counter, tot, vb) && threadIdx.x == 0) *out = tot[0];
  }
}

template <int P, bool DOT>
__global__ void __launch_bounds__(kThreads) k_stencil(Geo g, const double* __restrict__ tab,
                                                      const double* __restrict__ x, double* __restrict__ y,
                                                      double* partials, unsigned* counter, double* out) {
  stencil_body<P, DOT>(vblk_self(), g, tab, x, y, partials, counter, out);
}

// two operators on one vector in one pass: y1 = T1 x, y2 = T2 x
template <int P>
__device__ __forceinline__ void stencil2_body(VBlk vb, Geo g, const double* __restrict__ tab1,
                                                       const double* __restrict__ tab2, const double* __restrict__ x,
                                                       double* __restrict__ y1, double* __restrict__ y2) {
  const long long total = (long long)g.nxi * (P == 2 ? g.nxi : 1) * g.Ypad;
  for (long long t = (long long)vb.b * blockDim.x + threadIdx.x; t < total;
       t += (long long)vb.nb * blockDim.x) {
    Node nd = node_of<P>(g, t);
    const int cls = cls_of<P>(g, nd);
    y1[nd.idx] = stencil_at<P>(g, tab1, x, nd.idx, cls);
    y2[nd.idx] = stencil_at<P>(g, tab2, x, nd.idx, cls);
  }
}

template <int P>
__global__ void __launch_bounds__(kThreads) k_stencil2(Geo g, const double* __restrict__ tab1,
                                                       const double* __restrict__ tab2, const double* __restrict__ x,
                                                       double* __restrict__ y1, double* __restrict__ y2) {
  stencil2_body<P>(vblk_self(), g, tab1, tab2, x, y1, y2);
}

static long long interior_work(const Geo& g) {
  return (long long)g.nxi * (g.p == 2 ? g.nxi : 1) * g.Ypad;
}

void launch_stencil(dd_ctx* c, const double* tab, const double* x, double* y, cudaStream_t s) {
  const Geo& g = c->g;
  const long long w = interior_work(g);
  if (g.p == 1)
    (k_stencil<1, false><<<resident_grid(k_stencil<1, false>, w, kThreads), kThreads, 0, s>>>(g, tab, x, y, nullptr,
                                                                                              nullptr, nullptr),
     dd::note_launch());
  else
    (k_stencil<2, false><<<resident_grid(k_stencil<2, false>, w, kThreads), kThreads, 0, s>>>(g, tab, x, y, nullptr,
                                                                                              nullptr, nullptr),
     dd::note_launch());
  DD_CUDA(cudaGetLastError());
}

void launch_stencil2(dd_ctx* c, const double* tab1, const double* tab2, const double* x, double* y1, double* y2,
                     cudaStream_t s) {
  const Geo& g = c->g;
  const long long w = interior_work(g);
  if (g.p == 1)
    (k_stencil2<1><<<resident_grid(k_stencil2<1>, w, kThreads), kThreads, 0, s>>>(g, tab1, tab2, x, y1, y2),
     dd::note_launch());
  else
    (k_stencil2<2><<<resident_grid(k_stencil2<2>, w, kThreads), kThreads, 0, s>>>(g, tab1, tab2, x, y1, y2),
     dd::note_launch());
  DD_CUDA(cudaGetLastError());
}

void launch_stencil_dot(dd_ctx* c, const double* tab, const double* x, double* y, double* out,
                        unsigned* counter, cudaStream_t s) {
  const Geo& g = c->g;
  const long long w = interior_work(g);
  if (g.p == 1)
    (k_stencil<1, true><<<resident_grid(k_stencil<1, true>, w, kThreads), kThreads, 0, s>>>(g, tab, x, y, c->red,
                                                                                            counter, out),
     dd::note_launch());
  else
    (k_stencil<2, true><<<resident_grid(k_stencil<2, true>, w, kThreads), kThreads, 0, s>>>(g, tab, x, y, c->red,
                                                                                            counter, out),
     dd::note_launch());
  DD_CUDA(cudaGetLastError());
}

// ----------------------------------------------------------------------------------------
// Layout conversion between the ABI order (interior nodes, y fastest) and the padded order.
// ----------------------------------------------------------------------------------------
template <int P, bool TO_PAD>
__global__ void k_pad(Geo g, const double* __restrict__ src, double* __restrict__ dst) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < g.ndof;
       t += (long long)gridDim.x * blockDim.x) {
    const long long col = t / g.nyi;
    const int j = (int)(t - col * g.nyi);
    long long pidx;
    if (P == 1) pidx = (col + 1) * g.Ypad + j;
    else {
      const long long a1 = col / g.nxi + 1, a2 = col % g.nxi + 1;
      pidx = (a1 * g.ncx + a2) * g.Ypad + j;
    }
    if (TO_PAD) dst[pidx] = src[t];
    else dst[t] = src[pidx];
  }
}

void launch_pad(dd_ctx* c, const double* u, double* v, cudaStream_t s) {
  const Geo& g = c->g;
  const int nb = grid_blocks(g.ndof, kThreads);
  if (g.p == 1) (k_pad<1, true><<<nb, kThreads, 0, s>>>(g, u, v), dd::note_launch());
  else (k_pad<2, true><<<nb, kThreads, 0, s>>>(g, u, v), dd::note_launch());
  DD_CUDA(cudaGetLastError());
}

void launch_unpad(dd_ctx* c, const double* v, double* u, cudaStream_t s) {
  const Geo& g = c->g;
  const int nb = grid_blocks(g.ndof, kThreads);
  if (g.p == 1) (k_pad<1, false><<<nb, kThreads, 0, s>>>(g, v, u), dd::note_launch());
  else (k_pad<2, false><<<nb, kThreads, 0, s>>>(g, v, u), dd::note_launch());
  DD_CUDA(cudaGetLastError());
}

__global__ void k_check_finite(const double* __restrict__ v, long long n, int* flag) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n;
       t += (long long)gridDim.x * blockDim.x)
    if (!isfinite(v[t])) atomicOr(flag, 1);
}

void launch_check_finite(const double* v, long long n, int* flag, cudaStream_t s) {
  (k_check_finite<<<grid_blocks(n, kThreads), kThreads, 0, s>>>(v, n, flag), dd::note_launch());
  DD_CUDA(cudaGetLastError());
}

// ----------------------------------------------------------------------------------------
// PCG (Hestenes-Stiefel; flexible Polak-Ribiere beta when the preconditioner is rounded).
// The scalars live in PcgState on the device; every kernel returns at once when the
// iteration is marked done, so a fixed block of iterations can be replayed as a graph.
// ----------------------------------------------------------------------------------------

// r = b - A_sigma x, rr0 = (r, r), tol2 = rtol^2 rr0 (rtol^2 preset in tol2 by the host).
template <int P>
__device__ __forceinline__ void pcg_init_body(VBlk vb, Geo g, const double* __restrict__ tab,
                                                       const double* __restrict__ x,
                                                       const double* __restrict__ b, double* __restrict__ r,
                                                       PcgState* st, double* partials, unsigned* counter) {
  const long long total = (long long)g.nxi * (P == 2 ? g.nxi : 1) * g.Ypad;
  double acc[1] = {0.0};
  for (long long t = (long long)vb.b * blockDim.x + threadIdx.x; t < total;
       t += (long long)vb.nb * blockDim.x) {
    Node nd = node_of<P>(g, t);
    const int cls = cls_of<P>(g, nd);
    const double v = b[nd.idx] - stencil_at<P>(g, tab, x, nd.idx, cls);
    r[nd.idx] = v;
    acc[0] = fma(v, v, acc[0]);
  }
  double tot[1];
  if (grid_sum_last<1>(acc, partials, counter, tot, vb) && threadIdx.x == 0) {
    st->rr0 = tot[0];
    st->rr = tot[0];
    st->tol2 = st->tol2 * tot[0];
    st->iter = 0;
    st->beta = 0.0;
    st->status = 0;
    st->done = 0;
    if (!isfinite(tot[0])) { st->status = DD_ENAN; st->done = 1; }
    else if (tot[0] == 0.0) st->done = 1;
  }
}

template <int P>
__global__ void __launch_bounds__(kThreads) k_pcg_init(Geo g, const double* __restrict__ tab,
                                                       const double* __restrict__ x,
                                                       const double* __restrict__ b, double* __restrict__ r,
                                                       PcgState* st, double* partials, unsigned* counter) {
  pcg_init_body<P>(vblk_self(), g, tab, x, b, r, st, partials, counter);
}

void launch_pcg_init(dd_ctx* c, const double* b, cudaStream_t s) {
  const Geo& g = c->g;
  const int nb = grid_blocks(interior_work(g), kThreads);
  if (g.p == 1)
    (k_pcg_init<1><<<nb, kThreads, 0, s>>>(g, c->tabS, c->x, b, c->r, c->st, c->red, c->cnt + CNT_INIT), dd::note_launch());
  else
    (k_pcg_init<2><<<nb, kThreads, 0, s>>>(g, c->tabS, c->x, b, c->r, c->st, c->red, c->cnt + CNT_INIT), dd::note_launch());
  DD_CUDA(cudaGetLastError());
}

// p_k = z + beta p_{k-1} (whole padded vector; boundary columns and pads stay zero); the
// double buffer's index helpers p_prev / p_cur are in dd_common.cuh.

// x (when not null): the previous iteration's x += alpha_{k-1} p_{k-1}, deferred to this
// pass, which reads p_{k-1} anyway (see x_lag in dd_internal.h).
__global__ void __launch_bounds__(kThreads) k_pupdate(long long n, const double* __restrict__ z, double* pb0,
                                                      double* pb1, double* __restrict__ x, const PcgState* st) {
  if (st->done) return;
  const double beta = st->beta;
  const int k = st->iter;
  const double alpha = st->alpha;
  const bool upx = x != nullptr && k > 0;
  const double2* z2 = reinterpret_cast<const double2*>(z);
  const double2* pp = reinterpret_cast<const double2*>(p_prev(pb0, pb1, k));
  double2* pc = reinterpret_cast<double2*>(p_cur(pb0, pb1, k));
  double2* x2 = reinterpret_cast<double2*>(x);
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n / 2;
       t += (long long)gridDim.x * blockDim.x) {
    double2 a = z2[t], b = pp[t];
    if (upx) {
      double2 xv = x2[t];
      xv.x = fma(alpha, b.x, xv.x);
      xv.y = fma(alpha, b.y, xv.y);
      x2[t] = xv;
    }
    b.x = fma(beta, b.x, a.x);
    b.y = fma(beta, b.y, a.y);
    pc[t] = b;
  }
}

void launch_pupdate(dd_ctx* c, cudaStream_t s) {
  const long long n = c->g.plen;
  (k_pupdate<<<grid_blocks(n / 2, kThreads), kThreads, 0, s>>>(n, c->z, c->pb[0], c->pb[1], x_lag_target(c), c->st),
   dd::note_launch());
  DD_CUDA(cudaGetLastError());
}

// p = 1 fused K1: tiles of TC node columns plus one halo column per side are staged in
// shared memory as p_k = z + beta p_{k-1} (each value computed once per tile), written
// back for the tile's own columns, and the 9-point stencil q = A_sigma p_k and (p_k, q)
// are evaluated from shared memory.
constexpr int kFusedCols = 32;

// U2 = 2: each thread evaluates two nodes (e, e + blockDim) per pass, their 9-tap chains
// interleaved; the (p, q) partial is accumulated in the same node order as with U2 = 1, so the
// result is bit-identical.
template <int U2>
__device__ __forceinline__ void fused_pq_body(VBlk vb, Geo g, const double* __restrict__ tab,
                                              const double* __restrict__ z, double* pb0, double* pb1,
                                              double* __restrict__ q, double* __restrict__ x, PcgState* st,
                                              double* partials, unsigned* counter) {
  if (st->done) return;
  extern __shared__ double sp_raw[];
  double* sp = sp_raw + 1;   // one zero guard element on each side
  const int k = st->iter;
  const double beta = st->beta;
  const double alpha = st->alpha;   // alpha_{k-1}: this pass's last block overwrites it after all have read it
  const bool upx = x != nullptr && k > 0;
  const double* __restrict__ pp = p_prev(pb0, pb1, k);
  double* __restrict__ pc = p_cur(pb0, pb1, k);
  const int Y = g.Ypad, yl = g.ylog;
  const int ntiles = (g.nxi + kFusedCols - 1) / kFusedCols;
  if (threadIdx.x == 0) {
    sp_raw[0] = 0.0;
    sp_raw[(kFusedCols + 2) * Y + 1] = 0.0;
  }
  double acc[1] = {0.0};
  for (int tile = vb.b; tile < ntiles; tile += vb.nb) {
    const int a0 = 1 + tile * kFusedCols;
    const int own = min(kFusedCols, g.nxi - (a0 - 1));
    const int nload = (own + 2) << yl;
    const long long gbase = (long long)(a0 - 1) << yl;
    __syncthreads();
    const int nown = own << yl;
    for (int e = threadIdx.x; e < nload; e += blockDim.x) {
      // x is loaded beside p_{k-1} and z (one memory round trip per pass), stored for own nodes
      const bool mine = upx && e >= Y && e < Y + nown;
      const double pv = pp[gbase + e], zv = z[gbase + e];
      const double xv = mine ? x[gbase + e] : 0.0;
      sp[e] = fma(beta, pv, zv);
      if (mine) x[gbase + e] = fma(alpha, pv, xv);
    }
    if (threadIdx.x == 0) sp[nload] = 0.0;   // corner tap of the last (pad) slot of a partial tile
    __syncthreads();
    if (U2 == 1) {
      for (int e = threadIdx.x; e < nown; e += blockDim.x) {
        const int se = e + Y;
        const long long gi = gbase + se;
        const double pv = sp[se];
        pc[gi] = pv;
        const int col = a0 + (e >> yl), slot = e & (Y - 1);
        const int cls = (col % g.n) * Y + slot;
        double qv = 0.0;
#pragma unroll
        for (int dx = -1; dx <= 1; ++dx)
#pragma unroll
          for (int dy = -1; dy <= 1; ++dy)
            qv = fma(__ldg(tab + (size_t)((dx + 1) * 3 + (dy + 1)) * g.ncls + cls), sp[se + dx * Y + dy], qv);
        q[gi] = qv;
        acc[0] = fma(pv, qv, acc[0]);
      }
    } else {
      for (int e = threadIdx.x; e < nown; e += 2 * blockDim.x) {
        const int e1 = e + blockDim.x;
        const bool two = e1 < nown;
        const int f = two ? e1 : e;   // a valid node for the masked second chain
        const int se0 = e + Y, se1 = f + Y;
        const double pv0 = sp[se0], pv1 = sp[se1];
        const int cls0 = ((a0 + (e >> yl)) % g.n) * Y + (e & (Y - 1));
        const int cls1 = ((a0 + (f >> yl)) % g.n) * Y + (f & (Y - 1));
        double q0 = 0.0, q1 = 0.0;
#pragma unroll
        for (int dx = -1; dx <= 1; ++dx)
#pragma unroll
          for (int dy = -1; dy <= 1; ++dy) {
            const double* tt = tab + (size_t)((dx + 1) * 3 + (dy + 1)) * g.ncls;
            q0 = fma(__ldg(tt + cls0), sp[se0 + dx * Y + dy], q0);
            q1 = fma(__ldg(tt + cls1), sp[se1 + dx * Y + dy], q1);
          }
        pc[gbase + se0] = pv0;
        q[gbase + se0] = q0;
        acc[0] = fma(pv0, q0, acc[0]);
        if (two) {
          pc[gbase + se1] = pv1;
          q[gbase + se1] = q1;
          acc[0] = fma(pv1, q1, acc[0]);
        }
      }
    }
  }
  double tot[1];
  if (grid_sum_last<1>(acc, partials, counter, tot, vb) && threadIdx.x == 0) {
    const double pq = tot[0];
    st->pq = pq;
    if (!(pq > 0.0)) {
      st->status = isfinite(pq) ? DD_ENOTSPD : DD_ENAN;
      st->done = 1;
    } else {
      st->alpha = st->rho / pq;
    }
  }
}

// The same pass with q = A_sigma p evaluated in float pairs on the FP32 pipe: each staged p
// value is also split into (hi, lo) (integer operations), the 9 taps accumulate with the
// error-free product and sum (pair_fma) against the split table, and q = hi + lo in FP64.
// p_k, the (p, q) partial and everything else stay FP64; q differs from the FP64 stencil by
// up to 8.5 * 2^-47 (measured) times the sum of the taps' magnitudes.  Three FP64
// instructions per node (p update, q = hi + lo, the partial) instead of eleven.  The split table is class-major (a
// class's taps are five 16-byte loads), p_k is written back from the staging loop, and each
// thread evaluates two nodes (e, e + blockDim) per pass with their chains interleaved.
__device__ __forceinline__ void pair_taps(const float2* __restrict__ tab2, int cls, const float2* x, int Y,
                                          float& hs, float& ls) {
  const float4* tr = reinterpret_cast<const float4*>(tab2 + (size_t)cls * kPairTapStride);
  float t[18];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const float4 v = __ldg(tr + k);
    t[4 * k] = v.x; t[4 * k + 1] = v.y; t[4 * k + 2] = v.z; t[4 * k + 3] = v.w;
  }
  {
    const float4 v = __ldg(tr + 4);
    t[16] = v.x; t[17] = v.y;
  }
#pragma unroll
  for (int dx = -1; dx <= 1; ++dx)
#pragma unroll
    for (int dy = -1; dy <= 1; ++dy) {
      const int k = (dx + 1) * 3 + (dy + 1);
      const float2 xv = x[dx * Y + dy];
      pair_fma(t[2 * k], t[2 * k + 1], xv.x, xv.y, hs, ls);
    }
}

__device__ __forceinline__ void fused_pq_pairs_body(VBlk vb, Geo g, const float2* __restrict__ tab2,
                                                    const double* __restrict__ z, double* pb0, double* pb1,
                                                    double* __restrict__ q, double* __restrict__ x, PcgState* st,
                                                    double* partials, unsigned* counter) {
  if (st->done) return;
  extern __shared__ double sp_raw[];
  const int Y = g.Ypad, yl = g.ylog;
  const double alpha = st->alpha;   // alpha_{k-1}, read before this pass's last block replaces it
  const int nstage = (kFusedCols + 2) * Y + 2;
  float2* sp2_raw = reinterpret_cast<float2*>(sp_raw);
  float2* sp2 = sp2_raw + 1;   // one zero guard element on each side
  double* spd = sp_raw + nstage;   // the tile's own p values (FP64), for the partial
  const int k = st->iter;
  const double beta = st->beta;
  const bool upx = x != nullptr && k > 0;
  const double* __restrict__ pp = p_prev(pb0, pb1, k);
  double* __restrict__ pc = p_cur(pb0, pb1, k);
  const int ntiles = (g.nxi + kFusedCols - 1) / kFusedCols;
  if (threadIdx.x == 0) {
    sp2_raw[0] = make_float2(0.0f, 0.0f);
    sp2_raw[nstage - 1] = make_float2(0.0f, 0.0f);
  }
  const int cstep = blockDim.x >> yl;   // node columns per pass of the block (blockDim >= Y)
  double acc[1] = {0.0};
  for (int tile = vb.b; tile < ntiles; tile += vb.nb) {
    const int a0 = 1 + tile * kFusedCols;
    const int own = min(kFusedCols, g.nxi - (a0 - 1));
    const int nload = (own + 2) << yl;
    const int nown = own << yl;
    const long long gbase = (long long)(a0 - 1) << yl;
    __syncthreads();
    for (int e = threadIdx.x; e < nload; e += blockDim.x) {
      // x is loaded beside p_{k-1} and z (one memory round trip per pass), stored for own nodes
      const bool own_e = e >= Y && e < Y + nown;
      const double pprev = pp[gbase + e], zv = z[gbase + e];
      const double xv = (upx && own_e) ? x[gbase + e] : 0.0;
      const double pv = fma(beta, pprev, zv);
      sp2[e] = f64_split(pv);
      if (own_e) {
        pc[gbase + e] = pv;
        spd[e - Y] = pv;
        if (upx) x[gbase + e] = fma(alpha, pprev, xv);
      }
    }
    if (threadIdx.x == 0) sp2[nload] = make_float2(0.0f, 0.0f);   // corner tap of the last pad slot
    __syncthreads();
    // class column (a0 + e / Y) mod n, advanced by cstep columns per pass
    int cm = (a0 + (threadIdx.x >> yl)) % g.n;
    int cm1 = cm + cstep;
    while (cm1 >= g.n) cm1 -= g.n;
    for (int e = threadIdx.x; e < nown; e += 2 * blockDim.x) {
      const int e1 = e + blockDim.x;
      const bool two = e1 < nown;
      const int f = two ? e1 : e;   // a valid node for the masked second chain
      const int slot = e & (Y - 1);
      float h0 = 0.0f, l0 = 0.0f, h1 = 0.0f, l1 = 0.0f;
      pair_taps(tab2, cm * Y + slot, sp2 + e + Y, Y, h0, l0);
      pair_taps(tab2, cm1 * Y + slot, sp2 + f + Y, Y, h1, l1);
      const double q0 = f32_to_f64(h0) + f32_to_f64(l0);
      q[gbase + Y + e] = q0;
      acc[0] = fma(spd[e], q0, acc[0]);
      if (two) {
        const double q1 = f32_to_f64(h1) + f32_to_f64(l1);
        q[gbase + Y + e1] = q1;
        acc[0] = fma(spd[e1], q1, acc[0]);
      }
      cm += 2 * cstep;
      while (cm >= g.n) cm -= g.n;
      cm1 += 2 * cstep;
      while (cm1 >= g.n) cm1 -= g.n;
    }
  }
  double tot[1];
  if (grid_sum_last<1>(acc, partials, counter, tot, vb) && threadIdx.x == 0) {
    const double pq = tot[0];
    st->pq = pq;
    if (!(pq > 0.0)) {
      st->status = isfinite(pq) ? DD_ENOTSPD : DD_ENAN;
      st->done = 1;
    } else {
      st->alpha = st->rho / pq;
    }
  }
}

__global__ void __launch_bounds__(kThreads) k_fused_pq_pairs(Geo g, const float2* __restrict__ tab2,
                                                             const double* __restrict__ z, double* pb0, double* pb1,
                                                             double* __restrict__ q, double* __restrict__ x,
                                                             PcgState* st, double* partials, unsigned* counter) {
  pdl_enter();
  fused_pq_pairs_body(vblk_self(), g, tab2, z, pb0, pb1, q, x, st, partials, counter);
}

static size_t fused_pq_smem(int ypad, bool pairs) {
  const size_t n = (size_t)(kFusedCols + 2) * ypad + 2;
  return pairs ? n * sizeof(float2) + (size_t)kFusedCols * ypad * sizeof(double) : n * sizeof(double);
}

template <int U2>
__global__ void __launch_bounds__(kThreads) k_fused_pq(Geo g, const double* __restrict__ tab,
                                                       const double* __restrict__ z, double* pb0, double* pb1,
                                                       double* __restrict__ q, double* __restrict__ x, PcgState* st,
                                                       double* partials, unsigned* counter) {
  pdl_enter();
  fused_pq_body<U2>(vblk_self(), g, tab, z, pb0, pb1, q, x, st, partials, counter);
}

void launch_fused_pq(dd_ctx* c, cudaStream_t s) {
  const Geo& g = c->g;
  const int ntiles = (g.nxi + kFusedCols - 1) / kFusedCols;
  const int nb = ntiles < 152 * 6 ? ntiles : 152 * 6;
  const size_t smem = fused_pq_smem(g.Ypad, c->pq_pairs != 0);
  static PerDeviceOnce attr;   // once per device
  once_per_device(attr, [] {
    DD_CUDA(cudaFuncSetAttribute(k_fused_pq<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
    DD_CUDA(cudaFuncSetAttribute(k_fused_pq<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
    DD_CUDA(cudaFuncSetAttribute(k_fused_pq_pairs, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
  });
  const bool pdl = c->pdl != 0;
  if (c->pq_pairs) {
    launch_chain(k_fused_pq_pairs, dim3(nb), dim3(kThreads), smem, s, pdl, g, (const float2*)c->tabS2,
                 (const double*)c->z, c->pb[0], c->pb[1], c->q, x_lag_target(c), c->st, c->red, c->cnt + CNT_PQ);
    return;
  }
  // two nodes per thread and pass by default: 53.0 against 53.8 us per launch on the
  // L = 2048, h = 1/32 box, the same bits
  launch_chain(c->fused_pq_opt != 1 ? k_fused_pq<2> : k_fused_pq<1>, dim3(nb), dim3(kThreads), smem, s, pdl, g,
               (const double*)c->tabS, (const double*)c->z, c->pb[0], c->pb[1], c->q, x_lag_target(c), c->st,
               c->red, c->cnt + CNT_PQ);
}

// x[0..n) = v (start vectors of the convenience entry points)
__global__ void __launch_bounds__(kThreads) k_fill_value(long long n, double v, double* __restrict__ x) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x)
    x[t] = v;
}

void launch_fill(double* x, long long n, double v, cudaStream_t s) {
  (k_fill_value<<<grid_blocks(n, kThreads), kThreads, 0, s>>>(n, v, x), dd::note_launch());
  DD_CUDA(cudaGetLastError());
}

// q = A_sigma p, pq = (p, q), alpha = rho / pq.
template <int P>
__global__ void __launch_bounds__(kThreads) k_matvec_pq(Geo g, const double* __restrict__ tab, double* pb0,
                                                        double* pb1, double* __restrict__ q, PcgState* st,
                                                        double* partials, unsigned* counter) {
  if (st->done) return;
  const double* __restrict__ p = p_cur(pb0, pb1, st->iter);
  const long long total = (long long)g.nxi * (P == 2 ? g.nxi : 1) * g.Ypad;
  double acc[1] = {0.0};
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    Node nd = node_of<P>(g, t);
    const int cls = cls_of<P>(g, nd);
    const double v = stencil_at<P>(g, tab, p, nd.idx, cls);
    q[nd.idx] = v;
    acc[0] = fma(p[nd.idx], v, acc[0]);
  }
  double tot[1];
  if (grid_sum_last<1>(acc, partials, counter, tot) && threadIdx.x == 0) {
    const double pq = tot[0];
    st->pq = pq;
    if (!(pq > 0.0)) {
      st->status = isfinite(pq) ? DD_ENOTSPD : DD_ENAN;
      st->done = 1;
    } else {
      st->alpha = st->rho / pq;
    }
  }
}

void launch_matvec_pq(dd_ctx* c, cudaStream_t s) {
  const Geo& g = c->g;
  const int nb = grid_blocks(interior_work(g), kThreads);
  if (g.p == 1)
    (k_matvec_pq<1><<<nb, kThreads, 0, s>>>(g, c->tabS, c->pb[0], c->pb[1], c->q, c->st, c->red, c->cnt + CNT_PQ),
     dd::note_launch());
  else
    (k_matvec_pq<2><<<nb, kThreads, 0, s>>>(g, c->tabS, c->pb[0], c->pb[1], c->q, c->st, c->red, c->cnt + CNT_PQ),
     dd::note_launch());
  DD_CUDA(cudaGetLastError());
}

// p = 2 with float pairs: the p update also stores p split into (hi, lo) floats (integer
// operations, as f64_split), so that the 27 taps of every node read split values.
__global__ void __launch_bounds__(kThreads) k_pupdate_pairs(long long n, const double* __restrict__ z, double* pb0,
                                                            double* pb1, float2* __restrict__ p2,
                                                            double* __restrict__ x, const PcgState* st) {
  pdl_enter();
  if (st->done) return;
  const double beta = st->beta;
  const int k = st->iter;
  const double alpha = st->alpha;
  const bool upx = x != nullptr && k > 0;
  const double2* z2 = reinterpret_cast<const double2*>(z);
  const double2* pp = reinterpret_cast<const double2*>(p_prev(pb0, pb1, k));
  double2* pc = reinterpret_cast<double2*>(p_cur(pb0, pb1, k));
  double2* x2 = reinterpret_cast<double2*>(x);
  float4* ps = reinterpret_cast<float4*>(p2);
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n / 2;
       t += (long long)gridDim.x * blockDim.x) {
    double2 a = z2[t], b = pp[t];
    if (upx) {
      double2 xv = x2[t];
      xv.x = fma(alpha, b.x, xv.x);
      xv.y = fma(alpha, b.y, xv.y);
      x2[t] = xv;
    }
    b.x = fma(beta, b.x, a.x);
    b.y = fma(beta, b.y, a.y);
    pc[t] = b;
    const float2 u = f64_split(b.x), v = f64_split(b.y);
    ps[t] = make_float4(u.x, u.y, v.x, v.y);
  }
}

void launch_pupdate_pairs(dd_ctx* c, cudaStream_t s) {
  const long long n = c->g.plen;
  launch_chain(k_pupdate_pairs, dim3(grid_blocks(n / 2, kThreads)), dim3(kThreads), 0, s, c->pdl != 0, n,
               (const double*)c->z, c->pb[0], c->pb[1], c->p2, x_lag_target(c), (const PcgState*)c->st);
}

// p = 2: q = A_sigma p with the 27 taps in float pairs (split table, class-major, 14 aligned
// 16-byte loads per class; split p from the p update; error-free products and sums as in the
// p = 1 pass), q = hi + lo in FP64, pq = (p, q) and alpha in FP64.
__global__ void __launch_bounds__(kThreads) k_matvec_pq_pairs(Geo g, const float2* __restrict__ tab2,
                                                              const float2* __restrict__ p2, double* pb0,
                                                              double* pb1, double* __restrict__ q, PcgState* st,
                                                              double* partials, unsigned* counter) {
  pdl_enter();
  if (st->done) return;
  const double* __restrict__ p = p_cur(pb0, pb1, st->iter);
  const long long total = (long long)g.nxi * g.nxi * g.Ypad;
  const long long c1 = (long long)g.ncx * g.Ypad, c2 = g.Ypad;
  double acc[1] = {0.0};
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const Node nd = node_of<2>(g, t);
    const int cls = cls_of<2>(g, nd);
    const float4* tr = reinterpret_cast<const float4*>(tab2 + (size_t)cls * kPairTapStride3);
    const float2* x = p2 + nd.idx;
    float hs = 0.0f, ls = 0.0f;
#pragma unroll
    for (int k4 = 0; k4 < kPairTapStride3 / 2; ++k4) {
      const float4 tv = __ldg(tr + k4);
#pragma unroll
      for (int j = 0; j < 2; ++j) {
        const int tap = 2 * k4 + j;
        if (tap < 27) {
          const int d1 = tap / 9 - 1, d2 = (tap / 3) % 3 - 1, dy = tap % 3 - 1;
          const float2 xv = __ldg(x + d1 * c1 + d2 * c2 + dy);
          pair_fma(j ? tv.z : tv.x, j ? tv.w : tv.y, xv.x, xv.y, hs, ls);
        }
      }
    }
    const double qv = f32_to_f64(hs) + f32_to_f64(ls);
    q[nd.idx] = qv;
    acc[0] = fma(p[nd.idx], qv, acc[0]);
  }
  double tot[1];
  if (grid_sum_last<1>(acc, partials, counter, tot) && threadIdx.x == 0) {
    const double pq = tot[0];
    st->pq = pq;
    if (!(pq > 0.0)) {
      st->status = isfinite(pq) ? DD_ENOTSPD : DD_ENAN;
      st->done = 1;
    } else {
      st->alpha = st->rho / pq;
    }
  }
}

// The same pass tiled through shared memory.  The class of node (a1, a2, slot) is
// ((a1 mod n) n + a2 mod n) Ypad + slot, so a block that takes only planes a1 = r (mod n)
// needs n Ypad classes of the table: it stages that slice once (n Ypad rows of 28 float
// pairs), then walks its share of the residue's (plane, a2 tile) pairs; each tile (one plane,
// TA = blockDim / Ypad node columns, one node per thread) stages the split p of the planes
// a1 - 1 .. a1 + 1 over columns a2 - 1 .. a2 + TA, so every tap reads shared memory.  Each
// node's arithmetic is that of k_matvec_pq_pairs (the same q bits); the (p, q) partials are
// summed in another order.
constexpr int kTiledMaxClasses = 448;   // n Ypad <= 448: the table slice is at most 98 KB

__global__ void __launch_bounds__(kThreads) k_matvec_pq_pairs_tiled(Geo g, const float2* __restrict__ tab2,
                                                                    const float2* __restrict__ p2, double* pb0,
                                                                    double* pb1, double* __restrict__ q,
                                                                    PcgState* st, double* partials,
                                                                    unsigned* counter) {
  pdl_enter();
  if (st->done) return;
  extern __shared__ __align__(16) float4 smt[];
  const int Y = g.Ypad, yl = g.ylog, n = g.n;
  const int ncls_r = n * Y;                      // classes of one residue
  const int TA = (int)blockDim.x >> yl;          // node columns per tile (blockDim multiple of Y)
  float2* tabs = reinterpret_cast<float2*>(smt);                    // [ncls_r][28]
  float2* tile_raw = tabs + (size_t)ncls_r * kPairTapStride3;       // guard, [3][TA + 2][Y], guard
  float2* tile = tile_raw + 1;
  const int row = (TA + 2) * Y;                  // one plane's staged run
  const int nbr = (int)gridDim.x / n;            // blocks per residue
  const int r = (int)blockIdx.x % n, kb = (int)blockIdx.x / n;
  // the residue's table slice: classes (r n + m) Y + slot for m < n
  {
    const float4* src = reinterpret_cast<const float4*>(tab2 + (size_t)r * ncls_r * kPairTapStride3);
    float4* dst = smt;
    for (int e = threadIdx.x; e < ncls_r * (kPairTapStride3 / 2); e += blockDim.x) dst[e] = __ldg(src + e);
  }
  if (threadIdx.x == 0) {
    tile_raw[0] = make_float2(0.0f, 0.0f);
    tile_raw[3 * row + 1] = make_float2(0.0f, 0.0f);
  }
  const double* __restrict__ p = p_cur(pb0, pb1, st->iter);
  const int a1_first = (r == 0) ? n : r;
  const int nplanes = (a1_first <= g.nxi) ? (g.nxi - a1_first) / n + 1 : 0;
  const int ntile2 = (g.nxi + TA - 1) / TA;
  const long long ntiles = (long long)nplanes * ntile2;
  const long long c1 = (long long)g.ncx * Y;
  const int c = (int)threadIdx.x >> yl, slot = (int)threadIdx.x & (Y - 1);
  double acc[1] = {0.0};
  for (long long tt = kb; tt < ntiles; tt += nbr) {
    const int a1 = a1_first + n * (int)(tt / ntile2);
    const int a2_0 = 1 + TA * (int)(tt % ntile2);
    __syncthreads();   // the previous tile's taps are read (and, the first time, the table staged)
    for (int e = threadIdx.x; e < 3 * row; e += blockDim.x) {
      const int pl = e / row, w = e - pl * row;
      const int col = a2_0 - 1 + (w >> yl);
      tile[e] = (col <= g.nxi + 1) ? p2[(long long)(a1 - 1 + pl) * c1 + (long long)col * Y + (w & (Y - 1))]
                                   : make_float2(0.0f, 0.0f);
    }
    __syncthreads();
    const int a2 = a2_0 + c;
    if (a2 <= g.nxi) {
      const float4* tr = reinterpret_cast<const float4*>(tabs + (size_t)((a2 % n) * Y + slot) * kPairTapStride3);
      const float2* x = tile + row + (c + 1) * Y + slot;   // plane a1, column a2 (the centre of the taps)
      float hs = 0.0f, ls = 0.0f;
#pragma unroll
      for (int k4 = 0; k4 < kPairTapStride3 / 2; ++k4) {
        const float4 tv = tr[k4];
#pragma unroll
        for (int j = 0; j < 2; ++j) {
          const int tap = 2 * k4 + j;
          if (tap < 27) {
            const int d1 = tap / 9 - 1, d2 = (tap / 3) % 3 - 1, dy = tap % 3 - 1;
            const float2 xv = x[d1 * row + d2 * Y + dy];
            pair_fma(j ? tv.z : tv.x, j ? tv.w : tv.y, xv.x, xv.y, hs, ls);
          }
        }
      }
      const long long idx = ((long long)a1 * g.ncx + a2) * Y + slot;
      const double qv = f32_to_f64(hs) + f32_to_f64(ls);
      q[idx] = qv;
      acc[0] = fma(p[idx], qv, acc[0]);
    }
  }
  double tot[1];
  if (grid_sum_last<1>(acc, partials, counter, tot) && threadIdx.x == 0) {
    const double pq = tot[0];
    st->pq = pq;
    if (!(pq > 0.0)) {
      st->status = isfinite(pq) ? DD_ENOTSPD : DD_ENAN;
      st->done = 1;
    } else {
      st->alpha = st->rho / pq;
    }
  }
}

bool matvec_tiled_fits(const Geo& g) {
  return g.p == 2 && g.n * g.Ypad <= kTiledMaxClasses && g.Ypad <= kThreads && g.nxi >= g.n;
}

void launch_matvec_pq_pairs(dd_ctx* c, cudaStream_t s) {
  const Geo& g = c->g;
  if (g.p != 2) throw Error(DD_EINVAL, "the float-pair matvec pass is the p = 2 form");
  if (c->matvec_tiled && matvec_tiled_fits(g)) {
    const int TA = kThreads / g.Ypad;
    const size_t smem = sizeof(float2) * ((size_t)g.n * g.Ypad * kPairTapStride3 + 3 * (size_t)(TA + 2) * g.Ypad + 2);
    static PerDeviceOnce attr;
    once_per_device(attr, [] {
      DD_CUDA(cudaFuncSetAttribute(k_matvec_pq_pairs_tiled, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
    });
    int per_sm = 0;
    DD_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_matvec_pq_pairs_tiled, kThreads, smem));
    const int nbr = std::max(1, 152 * std::max(per_sm, 1) / g.n);   // blocks per residue
    launch_chain(k_matvec_pq_pairs_tiled, dim3(g.n * nbr), dim3(kThreads), smem, s, c->pdl != 0, g,
                 (const float2*)c->tabS2, (const float2*)c->p2, c->pb[0], c->pb[1], c->q, c->st, c->red,
                 c->cnt + CNT_PQ);
    return;
  }
  launch_chain(k_matvec_pq_pairs, dim3(resident_grid(k_matvec_pq_pairs, interior_work(g), kThreads)), dim3(kThreads),
               0, s, c->pdl != 0, g, (const float2*)c->tabS2, (const float2*)c->p2, c->pb[0], c->pb[1], c->q, c->st,
               c->red, c->cnt + CNT_PQ);
}

// x += alpha p, r -= alpha q, rr = (r, r); stop test ||r|| <= rtol ||r0|| (Sec. 4.1).  UPX
// false: x is left to the next iteration's p update (x_lag), so only r and q are read.
template <bool UPX>
__device__ __forceinline__ void xr_update_body(VBlk vb, long long n, double* pb0, double* pb1,
                                                        const double* __restrict__ q, double* __restrict__ x,
                                                        double* __restrict__ r, PcgState* st,
                                                        double* partials, unsigned* counter) {
  if (st->done) return;
  const double alpha = st->alpha;
  const double* __restrict__ p = p_cur(pb0, pb1, st->iter);
  const double2* p2 = reinterpret_cast<const double2*>(p);
  const double2* q2 = reinterpret_cast<const double2*>(q);
  double2* x2 = reinterpret_cast<double2*>(x);
  double2* r2 = reinterpret_cast<double2*>(r);
  double acc[1] = {0.0};
  for (long long t = (long long)vb.b * blockDim.x + threadIdx.x; t < n / 2;
       t += (long long)vb.nb * blockDim.x) {
    double2 qv = q2[t], rv = r2[t];
    if (UPX) {
      double2 pv = p2[t], xv = x2[t];
      xv.x = fma(alpha, pv.x, xv.x);
      xv.y = fma(alpha, pv.y, xv.y);
      x2[t] = xv;
    }
    rv.x = fma(-alpha, qv.x, rv.x);
    rv.y = fma(-alpha, qv.y, rv.y);
    r2[t] = rv;
    acc[0] = fma(rv.x, rv.x, acc[0]);
    acc[0] = fma(rv.y, rv.y, acc[0]);
  }
  double tot[1];
  if (grid_sum_last<1>(acc, partials, counter, tot, vb) && threadIdx.x == 0) {
    const double rr = tot[0];
    st->rr = rr;
    st->iter += 1;
    if (!isfinite(rr)) {
      st->status = DD_ENAN;
      st->done = 1;
    } else if (rr <= st->tol2) {
      st->done = 1;
    } else if (st->iter >= st->maxit) {
      st->status = DD_EMAXIT;
      st->done = 1;
    }
  }
}

template <bool UPX>
__global__ void __launch_bounds__(kThreads) k_xr_update(long long n, double* pb0, double* pb1,
                                                        const double* __restrict__ q, double* __restrict__ x,
                                                        double* __restrict__ r, PcgState* st,
                                                        double* partials, unsigned* counter) {
  pdl_enter();
  xr_update_body<UPX>(vblk_self(), n, pb0, pb1, q, x, r, st, partials, counter);
}

// After the last PCG iteration K: x += alpha_K p_K, the update the lagged scheme left for a
// next p update that does not run.  Not after a failed (p, q) or a non-finite iterate.
__global__ void __launch_bounds__(kThreads) k_x_final(long long n, const double* __restrict__ pb0,
                                                      const double* __restrict__ pb1, double* __restrict__ x,
                                                      const PcgState* st) {
  if (st->status != 0 && st->status != DD_EMAXIT) return;
  const double alpha = st->alpha;
  // after iteration K the counter is K + 1, and p_K sits where iteration K + 1 would read p_{k-1}
  const double2* p2 = reinterpret_cast<const double2*>(p_prev(const_cast<double*>(pb0), const_cast<double*>(pb1),
                                                                st->iter));
  double2* x2 = reinterpret_cast<double2*>(x);
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n / 2;
       t += (long long)gridDim.x * blockDim.x) {
    const double2 pv = p2[t];
    double2 xv = x2[t];
    xv.x = fma(alpha, pv.x, xv.x);
    xv.y = fma(alpha, pv.y, xv.y);
    x2[t] = xv;
  }
}

void launch_x_final(dd_ctx* c, cudaStream_t s) {
  const long long n = c->g.plen;
  (k_x_final<<<grid_blocks(n / 2, kThreads), kThreads, 0, s>>>(n, c->pb[0], c->pb[1], c->x, c->st),
   dd::note_launch());
  DD_CUDA(cudaGetLastError());
}

// The kernel takes 64 registers, so 4 blocks of 256 per SM are resident: one wave of 608
// blocks (22.5 us on the 2.03M-unknown L = 2048 box) instead of two of the default 1216
// (25.5 us).  (Two grid-stride steps per pass with their loads issued together took 26 us.)
static int xr_blocks(const dd_ctx* c) { return grid_blocks(c->g.plen / 2, kThreads, 4); }

void launch_xr_update(dd_ctx* c, cudaStream_t s) {
  const long long n = c->g.plen;
  launch_chain(x_lag_target(c) != nullptr ? k_xr_update<false> : k_xr_update<true>, dim3(xr_blocks(c)), dim3(kThreads),
               0, s, c->pdl != 0, n, c->pb[0], c->pb[1], (const double*)c->q, c->x, c->r, c->st, c->red,
               c->cnt + CNT_RR);
  DD_CUDA(cudaGetLastError());
}

// ----------------------------------------------------------------------------------------
// K5: prolong-sum of the preconditioner (Sec. 3.1):
//   z = sum_i R_i^T y_i + sum_i (D_i R_i psi) u0_i
// gathered per node from its (at most 2^p) owning subdomains in a fixed order, with the
// owners read from per-column tables; fused with (r, z) (and (q, z) for the flexible
// variant) and the beta update.  With rounded local inverses y is FP32, and the whole node
// value (owners' contributions and the coarse term, from FP32 copies of the weights and of
// u0) is formed in FP32 and widened exactly: the FP64 pipe then carries only the dot
// products.
//   mode 0: preconditioner only (no scalars); 1: PCG start (rho = (r,z), beta = 0);
//   2: PCG iteration (beta standard or flexible).
// ----------------------------------------------------------------------------------------
__device__ __forceinline__ double to_f64(float f) { return f32_to_f64(f); }
__device__ __forceinline__ double to_f64(double d) { return d; }
__device__ __forceinline__ float fma_t(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double fma_t(double a, double b, double c) { return fma(a, b, c); }

// Register budget: 32 per thread (8 blocks of 256 per SM) for p = 1, which fits it; 48
// (5 blocks) for p = 2, whose four owners per node spilled at 32 (on the L = 64, h = 1/16
// three-dimensional box: 987 -> 971 ms per ground state).  The FP64 p = 1 variant spills a
// little at 32 yet ran 4% faster there than at 48 without spills.
// ARITH (p = 1): the owners from p1_owners and their packed rows from the subdomain index
// (subdomain i is packed row i; its type is pt.x, pt.y or pt.z for the left end, the interior
// and the right end) instead of the two index tables -- the same values, without two levels of
// dependent loads per node (the host checks the formula against the tables at set-up).
// UPD (p = 1 iterations whose x update ran in the packing, launch_pack_xr): r_out = r - alpha q
// first (the same FMA as the separate x/r update, each node once), and the dots take that r.
template <int P, typename TY, bool RAS, int U, bool ARITH = false, bool UPD = false>
__device__ __forceinline__ void prolong_body(VBlk vb, Geo g, const int4* __restrict__ axown,
                                                      const int4* __restrict__ subrow,
                                                      const int4* __restrict__ colrow, const TY* __restrict__ Y,
                                                      const TY* __restrict__ wT, const TY* __restrict__ puT,
                                                      const TY* __restrict__ u0, int coarse,
                                                      const double* __restrict__ r, const double* __restrict__ q,
                                                      double* __restrict__ z, int mode, PcgState* st,
                                                      double* partials, unsigned* counter, int kpad = 0,
                                                      int4 pt = make_int4(0, 0, 0, 0), double* r_out = nullptr) {
  static_assert(!ARITH || P == 1, "closed-form owners are those of a p = 1 box");
  // p = 1 with the tables: colrow[a] holds, per owner of node column a, the offsets of its
  // packed row and type row at the column's local position (subrow[o] + local column * Ypad),
  // so a node's loads of Y, wT and u0 wait on one table load instead of two
  constexpr bool kColRow = (P == 1) && !ARITH;
  if (mode != 0 && st->done) return;
  const bool flex = (mode == 2) && st->flexible;
  const double alpha_r = UPD ? st->alpha : 0.0;
  const long long total = (long long)g.nxi * (P == 2 ? g.nxi : 1) * g.Ypad;
  const long long stride = (long long)vb.nb * blockDim.x;
  constexpr int NO = (P == 2) ? 4 : 2;  // owners per node at most; U nodes per thread and pass
  double acc[2] = {0.0, 0.0};
  for (long long t0 = (long long)vb.b * blockDim.x + threadIdx.x; t0 < total; t0 += U * stride) {
    // branch-free: out-of-range nodes and absent owners read valid addresses and are masked
    bool in[U], valid[U];
    Node nd[U];
    int4 A1[U], A2[U], CR[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const long long t = t0 + u * stride;
      in[u] = t < total;
      nd[u] = node_of<P>(g, in[u] ? t : 0);
      valid[u] = in[u] && nd[u].slot < g.nyi;
      A1[u] = ARITH ? p1_owners(g, nd[u].a1) : __ldg(axown + nd[u].a1);
      A2[u] = (P == 2) ? __ldg(axown + nd[u].a2) : make_int4(0, 0, -1, 0);
      CR[u] = kColRow ? __ldg(colrow + nd[u].a1) : make_int4(0, 0, 0, 0);
    }
    bool ok[U][NO];
    int sub[U][NO], loc[U][NO];
    int4 sr[U][NO];
#pragma unroll
    for (int u = 0; u < U; ++u)
#pragma unroll
      for (int e = 0; e < NO; ++e) {
        const int i = (P == 2) ? e >> 1 : e, k = (P == 2) ? e & 1 : 0;
        const int o1 = i ? A1[u].z : A1[u].x, l1 = i ? A1[u].w : A1[u].y;
        const int o2 = k ? A2[u].z : A2[u].x, l2 = k ? A2[u].w : A2[u].y;
        ok[u][e] = o1 >= 0 && (P == 1 || o2 >= 0);
        sub[u][e] = ok[u][e] ? ((P == 1) ? o1 : o1 * g.L + o2) : 0;
        if (kColRow) {   // the owner's packed row and type row, its local column included
          sr[u][e] = i ? make_int4(CR[u].z, CR[u].w, 1, 0) : make_int4(CR[u].x, CR[u].y, 1, 0);
          loc[u][e] = ok[u][e] ? nd[u].slot : 0;
          continue;
        }
        if (ARITH) {
          const int sb = sub[u][e];
          const int ty = sb == 0 ? pt.x : (sb == g.L - 1 ? pt.z : pt.y);
          sr[u][e] = make_int4(sb * kpad, ty * kpad, 1, 0);
        } else {
          sr[u][e] = __ldg(subrow + sub[u][e]);
        }
        loc[u][e] = ok[u][e] ? (((P == 1) ? l1 : l1 * sr[u][e].z + l2) * g.Ypad + nd[u].slot) : 0;
      }
    double rv[U], qv[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      rv[u] = (mode != 0) ? r[nd[u].idx] : 0.0;
      const double qq = (flex || UPD) ? q[nd[u].idx] : 0.0;
      if (UPD) {
        rv[u] = fma(-alpha_r, qq, rv[u]);
        if (in[u]) r_out[nd[u].idx] = rv[u];
      }
      qv[u] = flex ? qq : 0.0;
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      TY ys = (TY)0, cz = (TY)0;
#pragma unroll
      for (int e = 0; e < NO; ++e) {
        const size_t ry = (size_t)sr[u][e].x + loc[u][e], rw = (size_t)sr[u][e].y + loc[u][e];
        TY y = Y[ry];
        if (RAS) y = __ldg(puT + rw) * y;   // R_i^T D_i y_i
        const TY cw = coarse ? fma_t(__ldg(wT + rw), __ldg(u0 + sub[u][e]), cz) : cz;
        if (ok[u][e]) {
          ys += y;
          cz = cw;
        }
      }
      const double v = valid[u] ? to_f64(ys + cz) : 0.0;
      if (in[u]) {
        z[nd[u].idx] = v;
        if (mode != 0) {
          acc[0] = fma(rv[u], v, acc[0]);
          if (flex) acc[1] = fma(qv[u], v, acc[1]);
        }
      }
    }
  }
  if (mode == 0) return;
  double tot[2];
  if (grid_sum_last<2>(acc, partials, counter, tot, vb) && threadIdx.x == 0) {
    const double rz = tot[0];
    if (!isfinite(rz)) {
      st->status = DD_ENAN;
      st->done = 1;
      return;
    }
    if (mode == 1) {
      st->beta = 0.0;
    } else if (st->flexible) {
      st->beta = -tot[1] / st->pq;   // (z_{k+1}, r_{k+1} - r_k)/(z_k, r_k) = -(z_{k+1}, q_k)/pq_k
    } else {
      st->beta = rz / st->rho;
    }
    st->rho = rz;
    st->zq = tot[1];
  }
}

template <int P, typename TY, bool RAS, int U, bool ARITH = false, bool UPD = false>
__global__ void __launch_bounds__(kThreads, (P == 1 ? 8 : 5) / U) k_prolong(Geo g, const int4* __restrict__ axown,
                                                      const int4* __restrict__ subrow,
                                                      const int4* __restrict__ colrow, const TY* __restrict__ Y,
                                                      const TY* __restrict__ wT, const TY* __restrict__ puT,
                                                      const TY* __restrict__ u0, int coarse,
                                                      const double* __restrict__ r, const double* __restrict__ q,
                                                      double* __restrict__ z, int mode, PcgState* st,
                                                      double* partials, unsigned* counter, int kpad, int4 pt,
                                                      double* r_out) {
  pdl_enter();
  prolong_body<P, TY, RAS, U, ARITH, UPD>(vblk_self(), g, axown, subrow, colrow, Y, wT, puT, u0, coarse, r, q, z,
                                          mode, st, partials, counter, kpad, pt, r_out);
}

// nodes per thread and pass (each node's loads go out together, absent owners masked):
// measured on the L = 2048, h = 1/32 box, 24.7 / 31.5 / 42.4 us per launch for 1 / 2 / 4 (the register cost of
// more nodes takes away more resident warps than it adds loads in flight)
constexpr int kProlongU = 1;

void launch_prolong(dd_ctx* c, int mode, cudaStream_t s, double* zout, bool upd) {
  const Geo& g = c->g;
  const long long work = interior_work(g);
  const int coarse = c->grid.coarse;
  const bool f32 = (c->grid.precision != DD_PREC_FP64);
  double* z = zout != nullptr ? zout : c->z;
  const bool upd_r = upd && mode == 2;
#define DD_PROLONG_A(PP, TY, YP, W, PU, U0, RS, AR, UP)                                                          \
  launch_chain(k_prolong<PP, TY, RS, kProlongU, AR, UP>,                                                          \
               dim3(resident_grid(k_prolong<PP, TY, RS, kProlongU, AR, false>, work, kThreads)), dim3(kThreads), 0, \
               s, c->pdl != 0, g, (const int4*)c->axown, (const int4*)c->subrow, (const int4*)c->colrow,        \
               (const TY*)(YP),                                                                               \
               (const TY*)(W), (const TY*)(PU), (const TY*)(U0), coarse, (const double*)c->r,                    \
               (const double*)c->q, z, mode, c->st, c->red, c->cnt + CNT_RZ, c->kpad, c->ptypes,               \
               UP ? c->r : (double*)nullptr)
#define DD_PROLONG(PP, TY, YP, W, PU, U0, RS)                                    \
  do {                                                                           \
    if (PP == 1 && c->prolong_arith) DD_PROLONG_A(1, TY, YP, W, PU, U0, RS, true, false); \
    else DD_PROLONG_A(PP, TY, YP, W, PU, U0, RS, false, false);                 \
  } while (0)
#define DD_PROLONG_T(PP, RS)                                                          \
  do {                                                                                \
    if (f32) DD_PROLONG(PP, float, c->Y32, c->wT32, c->puT32, c->u0f, RS);           \
    else DD_PROLONG(PP, double, c->Y64, c->wT, c->puT, c->u0, RS);                    \
  } while (0)
  if (upd_r) {   // p = 1, rounded local inverses, AS (launch_pack_xr ran before)
    if (g.p != 1 || !f32 || c->ras) throw Error(DD_EINVAL, "the r update of the prolong-sum needs p = 1 and FP32 local results");
    if (c->prolong_arith) DD_PROLONG_A(1, float, c->Y32, c->wT32, c->puT32, c->u0f, false, true, true);
    else DD_PROLONG_A(1, float, c->Y32, c->wT32, c->puT32, c->u0f, false, false, true);
  } else if (c->ras) {
    if (g.p == 1) DD_PROLONG_T(1, true);
    else DD_PROLONG_T(2, true);
  } else {
    if (g.p == 1) DD_PROLONG_T(1, false);
    else DD_PROLONG_T(2, false);
  }
#undef DD_PROLONG_T
#undef DD_PROLONG
#undef DD_PROLONG_A
  DD_CUDA(cudaGetLastError());
}

// ----------------------------------------------------------------------------------------
// K7: outer step of the inverse iteration (Sec. 2).
//   normalize: given w (w1) and M w (w2): wMw = (w, Mw), s = sum w;
//              x = w / sqrt(wMw) (sign so that sum x > 0), Mx = Mw / sqrt(wMw)
//   residual : given A_sigma x (w3) and Mx (w2): mu = (x, A_sigma x);
//              ||A_sigma x - mu M x||^2 and ||M x||^2
// ----------------------------------------------------------------------------------------
__device__ __forceinline__ void outer_dots_body(VBlk vb, long long n, const double* __restrict__ w,
                                                         const double* __restrict__ Mw, OuterState* os,
                                                         double* partials, unsigned* counter) {
  double acc[2] = {0.0, 0.0};
  for (long long t = (long long)vb.b * blockDim.x + threadIdx.x; t < n;
       t += (long long)vb.nb * blockDim.x) {
    acc[0] = fma(w[t], Mw[t], acc[0]);
    acc[1] += w[t];
  }
  double tot[2];
  if (grid_sum_last<2>(acc, partials, counter, tot, vb) && threadIdx.x == 0) {
    os->wMw = tot[0];
    os->wsum = tot[1];
    if (!(tot[0] > 0.0)) {
      os->status = isfinite(tot[0]) ? DD_ENOTSPD : DD_ENAN;
      os->scale = 0.0;
    } else {
      os->scale = (tot[1] < 0.0 ? -1.0 : 1.0) / sqrt(tot[0]);
    }
  }
}

__global__ void __launch_bounds__(kThreads) k_outer_dots(long long n, const double* __restrict__ w,
                                                         const double* __restrict__ Mw, OuterState* os,
                                                         double* partials, unsigned* counter) {
  outer_dots_body(vblk_self(), n, w, Mw, os, partials, counter);
}

__device__ __forceinline__ void outer_scale_body(VBlk vb, long long n, double* __restrict__ x,
                                                          const double* __restrict__ w, double* __restrict__ Mw,
                                                          const OuterState* os) {
  const double s = os->scale;
  for (long long t = (long long)vb.b * blockDim.x + threadIdx.x; t < n;
       t += (long long)vb.nb * blockDim.x) {
    x[t] = s * w[t];
    Mw[t] *= s;
  }
}

__global__ void __launch_bounds__(kThreads) k_outer_scale(long long n, double* __restrict__ x,
                                                          const double* __restrict__ w, double* __restrict__ Mw,
                                                          const OuterState* os) {
  outer_scale_body(vblk_self(), n, x, w, Mw, os);
}

void launch_outer_normalize(dd_ctx* c, const double* w, double* Mw, double* xout, cudaStream_t s) {
  const long long n = c->g.plen;
  const int nb = grid_blocks(n, kThreads);
  (k_outer_dots<<<nb, kThreads, 0, s>>>(n, w, Mw, c->ost, c->red, c->cnt + CNT_OUTER0), dd::note_launch());
  (k_outer_scale<<<nb, kThreads, 0, s>>>(n, xout, w, Mw, c->ost), dd::note_launch());
  DD_CUDA(cudaGetLastError());
}

__device__ __forceinline__ void outer_res_body(VBlk vb, long long n, const double* __restrict__ Ax,
                                                        const double* __restrict__ Mx, OuterState* os,
                                                        double* partials, unsigned* counter, double* __restrict__ ro) {
  const double mu = os->xAx;
  double acc[2] = {0.0, 0.0};
  for (long long t = (long long)vb.b * blockDim.x + threadIdx.x; t < n;
       t += (long long)vb.nb * blockDim.x) {
    const double e = fma(-mu, Mx[t], Ax[t]);
    if (ro != nullptr) ro[t] = e;
    acc[0] = fma(e, e, acc[0]);
    acc[1] = fma(Mx[t], Mx[t], acc[1]);
  }
  double tot[2];
  if (grid_sum_last<2>(acc, partials, counter, tot, vb) && threadIdx.x == 0) {
    os->rr = tot[0];
    os->mm = tot[1];
  }
}

__global__ void __launch_bounds__(kThreads) k_outer_res(long long n, const double* __restrict__ Ax,
                                                        const double* __restrict__ Mx, OuterState* os,
                                                        double* partials, unsigned* counter, double* __restrict__ ro) {
  outer_res_body(vblk_self(), n, Ax, Mx, os, partials, counter, ro);
}

void launch_outer_residual(dd_ctx* c, const double* xe, const double* Mx, double* Ax, cudaStream_t s, double* ro) {
  // Ax = A_sigma x and xAx = (x, A_sigma x); then the residual norms (and the residual
  // A_sigma x - xAx M x = A x - rho M x itself when ro is given).
  launch_stencil_dot(c, c->tabS, xe, Ax, &c->ost->xAx, c->cnt + CNT_OUTER1, s);
  const long long n = c->g.plen;
  (k_outer_res<<<grid_blocks(n, kThreads), kThreads, 0, s>>>(n, Ax, Mx, c->ost, c->red, c->cnt + CNT_OUTER2, ro),
   dd::note_launch());
  DD_CUDA(cudaGetLastError());
}

void launch_outer_dots(dd_ctx* c, const double* w, const double* Mw, cudaStream_t s) {
  const long long n = c->g.plen;
  (k_outer_dots<<<grid_blocks(n, kThreads), kThreads, 0, s>>>(n, w, Mw, c->ost, c->red, c->cnt + CNT_OUTER0),
   dd::note_launch());
  DD_CUDA(cudaGetLastError());
}

// ----------------------------------------------------------------------------------------
// Gradients with respect to V at the cell quadrature points.  M_V is assembled from
// h^d W_q V_q N(z_q) N(z_q)^T on every box element, with V_q = V_cell_qp[e, q] on every copy
// of cell element e; so d(u^T M_V v)/dV_cell_qp[e, q] = sum over the copies of e of
// h^d W_q u_h(z_q) v_h(z_q).  Stage 1: partial sums over chunks of cells (cells in order);
// stage 2: the chunks in order (deterministic).
// ----------------------------------------------------------------------------------------
template <int P>
__global__ void __launch_bounds__(kThreads) k_qp_partial(Geo g, const double* __restrict__ u,
                                                         const double* __restrict__ v, int ny, int nq,
                                                         int cells_per_chunk, int nchunk, double* part) {
  constexpr int D = P + 1;
  const long long ncell_el = (long long)(P == 2 ? g.n * g.n : g.n) * ny;
  const long long per_chunk = ncell_el * nq;
  const long long total = per_chunk * nchunk;
  const int Q = g.Q;
  const long long ncells = (P == 2) ? (long long)g.L * g.L : g.L;
  double hd = 1.0;
  for (int k = 0; k < D; ++k) hd *= g.h;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const int ch = (int)(t / per_chunk);
    const long long r = t - (long long)ch * per_chunk;
    const long long e = r / nq;
    const int q = (int)(r - e * nq);
    // quadrature point (qx[, qx2], qy), qy fastest; element (ex[, ex2], ey), ey fastest
    int qa[3], ea[3];
    {
      int rq = q;
      for (int k = D - 1; k >= 0; --k) {
        qa[k] = rq % Q;
        rq /= Q;
      }
      long long re = e;
      ea[D - 1] = (int)(re % ny);
      re /= ny;
      for (int k = D - 2; k >= 0; --k) {
        ea[k] = (int)(re % g.n);
        re /= g.n;
      }
    }
    double wq = hd, nb[3][2];
    for (int k = 0; k < D; ++k) {
      const double xi = c_gpt[qa[k]];
      wq *= c_gwt[qa[k]];
      nb[k][0] = 1.0 - xi;
      nb[k][1] = xi;
    }
    const long long c0 = (long long)ch * cells_per_chunk;
    const long long c1 = min(ncells, c0 + cells_per_chunk);
    double acc = 0.0;
    for (long long cc = c0; cc < c1; ++cc) {
      const int cx1 = (P == 2) ? (int)(cc / g.L) : (int)cc;
      const int cx2 = (P == 2) ? (int)(cc % g.L) : 0;
      const int ex1 = cx1 * g.n + ea[0];
      const int ex2 = (P == 2) ? cx2 * g.n + ea[1] : 0;
      const int ey = ea[D - 1];
      double uh = 0.0, vh = 0.0;
#pragma unroll
      for (int b = 0; b < (1 << D); ++b) {
        // local node bits: x1 slowest, y fastest
        const int by = b & 1;
        const int b1 = (b >> (D - 1)) & 1;
        const int b2 = (P == 2) ? (b >> 1) & 1 : 0;
        const long long col = (P == 2) ? (long long)(ex1 + b1) * g.ncx + (ex2 + b2) : (long long)(ex1 + b1);
        const long long idx = col * g.Ypad + (ey + by - 1);   // slot -1 / nyi: zero pad or guard
        double nv = nb[0][b1] * nb[D - 1][by];
        if (P == 2) nv *= nb[1][b2];
        uh = fma(nv, u[idx], uh);
        vh = fma(nv, v[idx], vh);
      }
      acc = fma(uh, vh, acc);
    }
    part[t] = wq * acc;
  }
}

__global__ void __launch_bounds__(kThreads) k_qp_sum(long long n, int nchunk, const double* __restrict__ part,
                                                     double* out) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n;
       t += (long long)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int ch = 0; ch < nchunk; ++ch) s += part[(size_t)ch * n + t];
    out[t] = s;
  }
}

void launch_qp_product(dd_ctx* c, const double* u, const double* v, double* out, cudaStream_t s) {
  const Geo& g = c->g;
  const int ny = g.nyi + 1;
  int nq = 1;
  for (int k = 0; k < g.p + 1; ++k) nq *= g.Q;
  const long long ncell_el = (long long)(g.p == 2 ? g.n * g.n : g.n) * ny;
  const long long ncells = (g.p == 2) ? (long long)g.L * g.L : g.L;
  const long long per = ncell_el * nq;
  long long nchunk = (152LL * 2048 + per - 1) / per;
  nchunk = std::max(1LL, std::min(nchunk, ncells));
  const int cpc = (int)((ncells + nchunk - 1) / nchunk);
  nchunk = (ncells + cpc - 1) / cpc;
  if (c->qp_part_len < per * nchunk) {
    c->qp_part = (double*)dev_alloc(c, sizeof(double) * per * nchunk);
    c->qp_part_len = per * nchunk;
  }
  const long long total = per * nchunk;
  const int nb = (int)std::min<long long>((total + kThreads - 1) / kThreads, 152LL * 64);
  if (g.p == 1)
    (k_qp_partial<1><<<nb, kThreads, 0, s>>>(g, u, v, ny, nq, cpc, (int)nchunk, c->qp_part), dd::note_launch());
  else
    (k_qp_partial<2><<<nb, kThreads, 0, s>>>(g, u, v, ny, nq, cpc, (int)nchunk, c->qp_part), dd::note_launch());
  (k_qp_sum<<<grid_blocks(per, kThreads), kThreads, 0, s>>>(per, (int)nchunk, c->qp_part, out), dd::note_launch());
  DD_CUDA(cudaGetLastError());
}

// (a, b) over the padded vectors, deterministic; result in *out (device)
__global__ void __launch_bounds__(kThreads) k_dot(long long n, const double* __restrict__ a,
                                                  const double* __restrict__ b, double* out, double* partials,
                                                  unsigned* counter) {
  double acc[1] = {0.0};
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n;
       t += (long long)gridDim.x * blockDim.x)
    acc[0] = fma(a[t], b[t], acc[0]);
  double tot[1];
  if (grid_sum_last<1>(acc, partials, counter, tot) && threadIdx.x == 0) *out = tot[0];
}

// out = ca x + cb_scale * (*cb) y  (cb read on the device; out may alias x)
__global__ void __launch_bounds__(kThreads) k_axpby(long long n, double ca, const double* x, double cb_scale,
                                                    const double* cb, const double* y, double* out) {
  const double b = cb_scale * (cb != nullptr ? *cb : 1.0);
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n;
       t += (long long)gridDim.x * blockDim.x)
    out[t] = fma(b, y[t], ca * x[t]);
}

void launch_dot(dd_ctx* c, const double* a, const double* b, double* out, cudaStream_t s) {
  const long long n = c->g.plen;
  (k_dot<<<grid_blocks(n, kThreads), kThreads, 0, s>>>(n, a, b, out, c->red, c->cnt + CNT_GRAD), dd::note_launch());
  DD_CUDA(cudaGetLastError());
}

void launch_axpby(dd_ctx* c, double ca, const double* x, double cb_scale, const double* cb, const double* y,
                  double* out, cudaStream_t s) {
  const long long n = c->g.plen;
  (k_axpby<<<grid_blocks(n, kThreads), kThreads, 0, s>>>(n, ca, x, cb_scale, cb, y, out), dd::note_launch());
  DD_CUDA(cudaGetLastError());
}

void launch_tab_shift(dd_ctx* c, double shift, double* dst) {
  const long long n = (long long)c->g.ncls * c->g.ntap;
  (k_tabS<<<grid_blocks(n, kThreads), kThreads, 0, c->stream>>>(n, c->tabA, c->tabM, shift, dst), dd::note_launch());
  DD_CUDA(cudaGetLastError());
}


// ========================================================================================
// Batched launches (p = 1, rounded local inverses): the blocks of every problem's plain
// launch in one grid.  vmap[blockIdx.x] = {problem i, block b within problem i's launch};
// the block runs the plain kernel's body with the index b and count nb it has there, on
// problem i's buffers, so every problem's results are bit-identical to its plain launches.
// A problem whose eigen-iteration has stopped (active = 0) returns at once; so does every
// PCG kernel of a problem whose solve is done (its PcgState.done), as in a plain launch.
// ========================================================================================
static_assert(kMaxRedBlocksHost == kMaxRedBlocks, "host and device partial-slot counts differ");

__device__ __forceinline__ double* bvec(const BInst& I, int role) {
  if (role >= BV_LOP) return I.lop[role - BV_LOP];
  switch (role) {
    case BV_X: return I.x;
    case BV_R: return I.r;
    case BV_Z: return I.z;
    case BV_Q: return I.q;
    case BV_W1: return I.w1;
    case BV_W2: return I.w2;
    case BV_W3: return I.w3;
    default: return I.xe;
  }
}

// PcgState of a new solve: zero, then tol2 = rtol^2 (scaled by rr0 in pcg_init), maxit,
// flexible (what the host writes before a plain solve)
__global__ void kb_pcg_reset(const BInst* __restrict__ B, int n, double rtol2, int maxit) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n || !B[i].active) return;
  PcgState init;
  memset(&init, 0, sizeof(init));
  init.tol2 = rtol2;
  init.maxit = maxit;
  init.flexible = B[i].flexible;
  *B[i].st = init;
}

// x = 0 and both search-direction buffers = 0 (the plain solve's memsets)
__global__ void __launch_bounds__(kThreads) kb_zero_pcg(const BInst* __restrict__ B, const int2* __restrict__ vmap) {
  const int2 m = vmap[blockIdx.x];
  const BInst& I = B[m.x];
  if (!I.active) return;
  const long long n = I.g.plen;
  for (long long t = (long long)m.y * blockDim.x + threadIdx.x; t < n; t += (long long)I.nb_vec * blockDim.x) {
    I.x[t] = 0.0;
    I.pb0[t] = 0.0;
    I.pb1[t] = 0.0;
  }
}

__global__ void __launch_bounds__(kThreads, 8) kb_pcg_init(const BInst* __restrict__ B, const int2* __restrict__ vmap,
                                                        int b_role) {
  const int2 m = vmap[blockIdx.x];
  const BInst& I = B[m.x];
  if (!I.active) return;
  pcg_init_body<1>(VBlk{m.y, I.nb_init}, I.g, I.tabS, I.x, bvec(I, b_role), I.r, I.st, I.red, I.cnt + CNT_INIT);
}

template <bool PAIRS>
__global__ void __launch_bounds__(kThreads, 6) kb_fused_pq(const BInst* __restrict__ B, const int2* __restrict__ vmap) {
  const int2 m = vmap[blockIdx.x];
  const BInst& I = B[m.x];
  if (!I.active) return;
  if (PAIRS)
    fused_pq_pairs_body(VBlk{m.y, I.nb_fused}, I.g, I.tabS2, I.z, I.pb0, I.pb1, I.q, nullptr, I.st, I.red,
                        I.cnt + CNT_PQ);
  else
    fused_pq_body<2>(VBlk{m.y, I.nb_fused}, I.g, I.tabS, I.z, I.pb0, I.pb1, I.q, nullptr, I.st, I.red,
                     I.cnt + CNT_PQ);
}

__global__ void __launch_bounds__(kThreads) kb_xr_update(const BInst* __restrict__ B, const int2* __restrict__ vmap) {
  const int2 m = vmap[blockIdx.x];
  const BInst& I = B[m.x];
  if (!I.active) return;
  xr_update_body<true>(VBlk{m.y, I.nb_xr}, I.g.plen, I.pb0, I.pb1, I.q, I.x, I.r, I.st, I.red, I.cnt + CNT_RR);
}

template <bool ARITH, bool UPD>
__global__ void __launch_bounds__(kThreads, 8 / kProlongU) kb_prolong(const BInst* __restrict__ B,
                                                                      const int2* __restrict__ vmap, int mode) {
  const int2 m = vmap[blockIdx.x];
  const BInst& I = B[m.x];
  if (!I.active) return;
  prolong_body<1, float, false, kProlongU, ARITH, UPD>(VBlk{m.y, I.nb_prolong}, I.g, I.axown, I.subrow, I.colrow, I.Y32,
                                                       I.wT32, I.puT32, I.u0f, I.coarse, I.r, I.q, I.z, mode, I.st,
                                                       I.red, I.cnt + CNT_RZ, I.kpad, I.ptypes, UPD ? I.r : nullptr);
}

__global__ void __launch_bounds__(kThreads) kb_stencil(const BInst* __restrict__ B, const int2* __restrict__ vmap,
                                                       int mass, int x_role, int y_role) {
  const int2 m = vmap[blockIdx.x];
  const BInst& I = B[m.x];
  if (!I.active) return;
  stencil_body<1, false>(VBlk{m.y, I.nb_st}, I.g, mass ? I.tabM : I.tabS, bvec(I, x_role), bvec(I, y_role), nullptr,
                         nullptr, nullptr);
}

// y = A_sigma x and (x, A_sigma x) into the outer state (the plain outer residual's first pass)
__global__ void __launch_bounds__(kThreads, 6) kb_stencil_dot(const BInst* __restrict__ B, const int2* __restrict__ vmap,
                                                           int x_role, int y_role) {
  const int2 m = vmap[blockIdx.x];
  const BInst& I = B[m.x];
  if (!I.active) return;
  stencil_body<1, true>(VBlk{m.y, I.nb_sdot}, I.g, I.tabS, bvec(I, x_role), bvec(I, y_role), I.red,
                        I.cnt + CNT_OUTER1, &I.ost->xAx);
}

__global__ void __launch_bounds__(kThreads, 8) kb_outer_dots(const BInst* __restrict__ B, const int2* __restrict__ vmap,
                                                          int w_role, int mw_role) {
  const int2 m = vmap[blockIdx.x];
  const BInst& I = B[m.x];
  if (!I.active) return;
  outer_dots_body(VBlk{m.y, I.nb_vec}, I.g.plen, bvec(I, w_role), bvec(I, mw_role), I.ost, I.red,
                  I.cnt + CNT_OUTER0);
}

__global__ void __launch_bounds__(kThreads) kb_outer_scale(const BInst* __restrict__ B, const int2* __restrict__ vmap,
                                                           int x_role, int w_role, int mw_role) {
  const int2 m = vmap[blockIdx.x];
  const BInst& I = B[m.x];
  if (!I.active) return;
  outer_scale_body(VBlk{m.y, I.nb_vec}, I.g.plen, bvec(I, x_role), bvec(I, w_role), bvec(I, mw_role), I.ost);
}

__global__ void __launch_bounds__(kThreads, 8) kb_outer_res(const BInst* __restrict__ B, const int2* __restrict__ vmap,
                                                         int ax_role, int mx_role) {
  const int2 m = vmap[blockIdx.x];
  const BInst& I = B[m.x];
  if (!I.active) return;
  outer_res_body(VBlk{m.y, I.nb_vec}, I.g.plen, bvec(I, ax_role), bvec(I, mx_role), I.ost, I.red,
                 I.cnt + CNT_OUTER2, nullptr);
}

// every problem's PCG state marked done, whatever its active flag: the tiles of the grouped
// contraction (which read only that flag) then skip problems that have not joined yet
__global__ void kb_mark_done(const BInst* __restrict__ B, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) B[i].st->done = 1;
}

void launch_b_mark_done(const BInst* B, int n, cudaStream_t s) {
  (kb_mark_done<<<(n + 127) / 128, 128, 0, s>>>(B, n), dd::note_launch());
  DD_CUDA(cudaGetLastError());
}

__global__ void kb_gather(const BInst* __restrict__ B, int n, BStat* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const BInst& I = B[i];
  BStat o;
  o.pcg_done = I.st->done;
  o.pcg_status = I.st->status;
  o.pcg_iter = I.st->iter;
  o.active = I.active;
  o.xAx = I.ost->xAx;
  o.rr = I.ost->rr;
  o.mm = I.ost->mm;
  o.outer_status = I.ost->status;
  o.lop_status = I.lst != nullptr ? I.lst->status : 0;
  o.theta = I.lst != nullptr ? I.lst->theta : 0.0;
  o.lop_rr = I.lst != nullptr ? I.lst->rr : 0.0;
  o.lop_mm = I.lst != nullptr ? I.lst->mm : 0.0;
  out[i] = o;
}

// layout conversion between a user vector (ABI order) and a role vector (padded), p = 1
template <bool TO_PAD, bool ACTIVE_ONLY = false>
__global__ void __launch_bounds__(kThreads) kb_pad(const BInst* __restrict__ B, const int2* __restrict__ vmap,
                                                   const double* const* __restrict__ user_in,
                                                   double* const* __restrict__ user_out, int role) {
  const int2 m = vmap[blockIdx.x];
  const BInst& I = B[m.x];
  if (ACTIVE_ONLY && !I.active) return;
  const Geo& g = I.g;
  double* pv = bvec(I, role);
  for (long long t = (long long)m.y * blockDim.x + threadIdx.x; t < g.ndof; t += (long long)I.nb_vec * blockDim.x) {
    const long long col = t / g.nyi;
    const int j = (int)(t - col * g.nyi);
    const long long pidx = (col + 1) * g.Ypad + j;
    if (TO_PAD) pv[pidx] = user_in[m.x][t];
    else user_out[m.x][t] = pv[pidx];
  }
}

__global__ void __launch_bounds__(kThreads) kb_zero_roles(const BInst* __restrict__ B, const int2* __restrict__ vmap,
                                                          int first_role, int nroles) {
  const int2 m = vmap[blockIdx.x];
  const BInst& I = B[m.x];
  if (!I.active) return;
  const long long n = I.g.plen;
  for (int k = 0; k < nroles; ++k) {
    double* v = bvec(I, first_role + k);
    for (long long t = (long long)m.y * blockDim.x + threadIdx.x; t < n; t += (long long)I.nb_vec * blockDim.x)
      v[t] = 0.0;
  }
}

__global__ void kb_set_entry(const BInst* __restrict__ B, int n, int role, long long idx, double val) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n && B[i].active) bvec(B[i], role)[idx] = val;
}

__global__ void __launch_bounds__(kThreads) kb_stencil2(const BInst* __restrict__ B, const int2* __restrict__ vmap,
                                                        int x_role, int ys_role, int ym_role) {
  const int2 m = vmap[blockIdx.x];
  const BInst& I = B[m.x];
  if (!I.active) return;
  stencil2_body<1>(VBlk{m.y, I.nb_st2}, I.g, I.tabS, I.tabM, bvec(I, x_role), bvec(I, ys_role), bvec(I, ym_role));
}

__global__ void __launch_bounds__(kThreads, 8) kb_outer_res_ro(const BInst* __restrict__ B, const int2* __restrict__ vmap,
                                                            int ax_role, int mx_role, int ro_role) {
  const int2 m = vmap[blockIdx.x];
  const BInst& I = B[m.x];
  if (!I.active) return;
  outer_res_body(VBlk{m.y, I.nb_vec}, I.g.plen, bvec(I, ax_role), bvec(I, mx_role), I.ost, I.red,
                 I.cnt + CNT_OUTER2, ro_role == BV_NONE ? nullptr : bvec(I, ro_role));
}

void batch_grid_sizes(const dd_ctx* c, BInst* I) {
  const Geo& g = c->g;
  const long long w = interior_work(g);
  const int ntiles = (g.nxi + kFusedCols - 1) / kFusedCols;
  I->nb_init = grid_blocks(w, kThreads);
  I->nb_fused = ntiles < 152 * 6 ? ntiles : 152 * 6;
  I->nb_xr = xr_blocks(c);
  I->nb_prolong = c->prolong_arith ? resident_grid(k_prolong<1, float, false, kProlongU, true>, w, kThreads)
                                    : resident_grid(k_prolong<1, float, false, kProlongU, false>, w, kThreads);
  I->nb_sdot = resident_grid(k_stencil<1, true>, w, kThreads);
  I->nb_st = resident_grid(k_stencil<1, false>, w, kThreads);
  I->nb_vec = grid_blocks(g.plen, kThreads);
  I->nb_st2 = resident_grid(k_stencil2<1>, w, kThreads);
}

void launch_b_zero_roles(const BInst* B, const int2* vmap, int nvb, int first_role, int nroles, cudaStream_t s) {
  (kb_zero_roles<<<nvb, kThreads, 0, s>>>(B, vmap, first_role, nroles), dd::note_launch());
  DD_CUDA(cudaGetLastError());
}

void launch_b_set_entry(const BInst* B, int n, int role, long long idx, double val, cudaStream_t s) {
  (kb_set_entry<<<(n + 127) / 128, 128, 0, s>>>(B, n, role, idx, val), dd::note_launch());
  DD_CUDA(cudaGetLastError());
}

void launch_b_stencil_role(const BInst* B, const int2* vmap, int nvb, int mass, int x_role, int y_role,
                           cudaStream_t s) {
  launch_b_stencil(B, vmap, nvb, mass, x_role, y_role, s);
}

void launch_b_stencil2(const BInst* B, const int2* vmap_st2, int nvb, int x_role, int ys_role, int ym_role,
                       cudaStream_t s) {
  (kb_stencil2<<<nvb, kThreads, 0, s>>>(B, vmap_st2, x_role, ys_role, ym_role), dd::note_launch());
  DD_CUDA(cudaGetLastError());
}

void launch_b_outer_res_ro(const BInst* B, const int2* vmap, int nvb, int ax_role, int mx_role, int ro_role,
                           cudaStream_t s) {
  (kb_outer_res_ro<<<nvb, kThreads, 0, s>>>(B, vmap, ax_role, mx_role, ro_role), dd::note_launch());
  DD_CUDA(cudaGetLastError());
}

void launch_b_pcg_reset(const BInst* B, int n, double rtol2, int maxit, cudaStream_t s) {
  (kb_pcg_reset<<<(n + 127) / 128, 128, 0, s>>>(B, n, rtol2, maxit), dd::note_launch());
  DD_CUDA(cudaGetLastError());
}

void launch_b_zero_pcg(const BInst* B, const int2* vmap, int nvb, cudaStream_t s) {
  (kb_zero_pcg<<<nvb, kThreads, 0, s>>>(B, vmap), dd::note_launch());
  DD_CUDA(cudaGetLastError());
}

void launch_b_pcg_init(const BInst* B, const int2* vmap, int nvb, int b_role, cudaStream_t s) {
  (kb_pcg_init<<<nvb, kThreads, 0, s>>>(B, vmap, b_role), dd::note_launch());
  DD_CUDA(cudaGetLastError());
}

void launch_b_fused_pq(const BInst* B, const int2* vmap, int nvb, int ypad, bool pairs, cudaStream_t s) {
  const size_t smem = fused_pq_smem(ypad, pairs);
  static PerDeviceOnce attr;
  once_per_device(attr, [] {
    DD_CUDA(cudaFuncSetAttribute(kb_fused_pq<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
    DD_CUDA(cudaFuncSetAttribute(kb_fused_pq<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
  });
  if (pairs) (kb_fused_pq<true><<<nvb, kThreads, smem, s>>>(B, vmap), dd::note_launch());
  else (kb_fused_pq<false><<<nvb, kThreads, smem, s>>>(B, vmap), dd::note_launch());
  DD_CUDA(cudaGetLastError());
}

void launch_b_xr_update(const BInst* B, const int2* vmap, int nvb, cudaStream_t s) {
  (kb_xr_update<<<nvb, kThreads, 0, s>>>(B, vmap), dd::note_launch());
  DD_CUDA(cudaGetLastError());
}

void launch_b_prolong(const BInst* B, const int2* vmap, int nvb, int mode, bool arith, bool upd, cudaStream_t s) {
  if (upd && mode == 2) {
    if (arith) (kb_prolong<true, true><<<nvb, kThreads, 0, s>>>(B, vmap, mode), dd::note_launch());
    else (kb_prolong<false, true><<<nvb, kThreads, 0, s>>>(B, vmap, mode), dd::note_launch());
  } else {
    if (arith) (kb_prolong<true, false><<<nvb, kThreads, 0, s>>>(B, vmap, mode), dd::note_launch());
    else (kb_prolong<false, false><<<nvb, kThreads, 0, s>>>(B, vmap, mode), dd::note_launch());
  }
  DD_CUDA(cudaGetLastError());
}

void launch_b_stencil(const BInst* B, const int2* vmap, int nvb, int mass, int x_role, int y_role, cudaStream_t s) {
  (kb_stencil<<<nvb, kThreads, 0, s>>>(B, vmap, mass, x_role, y_role), dd::note_launch());
  DD_CUDA(cudaGetLastError());
}

void launch_b_stencil_dot(const BInst* B, const int2* vmap, int nvb, int x_role, int y_role, cudaStream_t s) {
  (kb_stencil_dot<<<nvb, kThreads, 0, s>>>(B, vmap, x_role, y_role), dd::note_launch());
  DD_CUDA(cudaGetLastError());
}

void launch_b_outer_normalize(const BInst* B, const int2* vmap, int nvb, int w_role, int mw_role, int x_role,
                              cudaStream_t s) {
  (kb_outer_dots<<<nvb, kThreads, 0, s>>>(B, vmap, w_role, mw_role), dd::note_launch());
  (kb_outer_scale<<<nvb, kThreads, 0, s>>>(B, vmap, x_role, w_role, mw_role), dd::note_launch());
  DD_CUDA(cudaGetLastError());
}

void launch_b_outer_dots_roles(const BInst* B, const int2* vmap, int nvb, int w_role, int mw_role, cudaStream_t s) {
  (kb_outer_dots<<<nvb, kThreads, 0, s>>>(B, vmap, w_role, mw_role), dd::note_launch());
  DD_CUDA(cudaGetLastError());
}

void launch_b_outer_res(const BInst* B, const int2* vmap, int nvb, int ax_role, int mx_role, cudaStream_t s) {
  (kb_outer_res<<<nvb, kThreads, 0, s>>>(B, vmap, ax_role, mx_role), dd::note_launch());
  DD_CUDA(cudaGetLastError());
}

void launch_b_gather(const BInst* B, int n, BStat* out, cudaStream_t s) {
  (kb_gather<<<(n + 127) / 128, 128, 0, s>>>(B, n, out), dd::note_launch());
  DD_CUDA(cudaGetLastError());
}

void launch_b_unpad(const BInst* B, const int2* vmap, int nvb, int src_role, double* const* dst, cudaStream_t s) {
  (kb_pad<false><<<nvb, kThreads, 0, s>>>(B, vmap, nullptr, dst, src_role), dd::note_launch());
  DD_CUDA(cudaGetLastError());
}

void launch_b_unpad_active(const BInst* B, const int2* vmap, int nvb, int src_role, double* const* dst,
                           cudaStream_t s) {
  (kb_pad<false, true><<<nvb, kThreads, 0, s>>>(B, vmap, nullptr, dst, src_role), dd::note_launch());
  DD_CUDA(cudaGetLastError());
}

void launch_b_pad(const BInst* B, const int2* vmap, int nvb, const double* const* src, int dst_role, cudaStream_t s) {
  (kb_pad<true, true><<<nvb, kThreads, 0, s>>>(B, vmap, src, nullptr, dst_role), dd::note_launch());
  DD_CUDA(cudaGetLastError());
}
}  // namespace dd

// ------------------------------------------------------------------------------------------
// Self-test of the integer-pipe precision conversions used by the mixed form (no paper
// counterpart): kind 0 rounds doubles to BF16 bits, kind 1 to TF32, kind 2 widens floats.
// ------------------------------------------------------------------------------------------
namespace dd {
__global__ void k_convert_test(int kind, long long n, const void* __restrict__ in, void* __restrict__ out) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
    if (kind == 0) static_cast<unsigned short*>(out)[t] = f64_to_bf16_bits(static_cast<const double*>(in)[t]);
    else if (kind == 1) static_cast<float*>(out)[t] = f64_to_tf32(static_cast<const double*>(in)[t]);
    else static_cast<double*>(out)[t] = f32_to_f64(static_cast<const float*>(in)[t]);
  }
}
}  // namespace dd

extern "C" int dd_convert_test(int kind, long long n, const void* in_host, void* out_host) {
  using namespace dd;
  if (kind < 0 || kind > 2 || n < 1 || !in_host || !out_host) return DD_EINVAL;
  const size_t in_b = (size_t)n * (kind == 2 ? 4 : 8), out_b = (size_t)n * (kind == 0 ? 2 : (kind == 1 ? 4 : 8));
  void *din = nullptr, *dout = nullptr;
  int rc = DD_OK;
  try {
    DD_CUDA(cudaMalloc(&din, in_b));
    DD_CUDA(cudaMalloc(&dout, out_b));
    DD_CUDA(cudaMemcpy(din, in_host, in_b, cudaMemcpyHostToDevice));
    (k_convert_test<<<grid_blocks(n, kThreads), kThreads>>>(kind, n, din, dout), dd::note_launch());
    DD_CUDA(cudaGetLastError());
    DD_CUDA(cudaMemcpy(out_host, dout, out_b, cudaMemcpyDeviceToHost));
  } catch (const Error& e) {
    rc = e.code;
  }
  if (din) cudaFree(din);
  if (dout) cudaFree(dout);
  return rc;
}
