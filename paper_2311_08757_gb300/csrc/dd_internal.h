// Internal declarations of the ddeig library: geometry, context, kernel launchers.
//
// Device data layout ("padded layout"): a box vector is stored over ALL node columns,
// boundary columns included, with Ypad >= ny slots per column:
//     index(col, slot) = col * Ypad + slot,  col = a (p = 1) or a1 (Ln + 1) + a2 (p = 2),
//     slot = j - 1 for the interior y-nodes j = 1..ny-1; slots ny-1..Ypad-1 are zero
//     (Ypad is the power of two >= ny, so index arithmetic is shifts and masks).
// Boundary columns (a = 0, a = Ln) and pad slots are kept at zero by every kernel, so
// the homogeneous Dirichlet condition (H^1_0, Sec. 1) needs no branch in the stencil:
// the neighbours of a node next to the boundary read zeros.  The corner taps of the first
// and last interior nodes reach one element outside [0, plen); every padded vector is
// allocated with a zeroed guard band on both sides for them.
#pragma once

#include <cuda_runtime.h>
#include <cstdint>
#include <cstddef>
#include <string>
#include <vector>

#include "../../include/ddeig.h"

namespace dd {

constexpr int kMaxQ = 4;
constexpr int kMaxTypes = 16;

// Geometry shared by host and device (passed by value to kernels).
struct Geo {
  int p;        // 1 or 2
  int L, n, ny, nyi;   // nyi = ny - 1 interior y nodes
  int delta, Q;
  int Ypad;     // slots per column: the power of two >= max(ny, 4)
  int ylog;     // log2(Ypad)
  int ncx;      // node columns per x axis incl. boundary = L n + 1
  int nxi;      // interior nodes per x axis = L n - 1
  long long ncol;   // ncx^p
  long long plen;   // ncol * Ypad  (padded vector length)
  long long ndof;   // nxi^p * nyi
  int nsub;     // L^p
  int ntap;     // 9 or 27
  int ncls;     // n^p * Ypad stencil classes
  double h;
};

// Per-axis subdomain geometry: subdomain i (0-based) covers interior node columns
// lo(i)..hi(i) along an x axis (Sec. 3.1: open overlapping boxes clipped at the box).
__host__ __device__ inline int ax_lo(const Geo& g, int i) {
  int v = i * g.n - g.delta + 1;
  return v < 1 ? 1 : v;
}
__host__ __device__ inline int ax_hi(const Geo& g, int i) {
  int v = (i + 1) * g.n + g.delta - 1;
  int m = g.L * g.n - 1;
  return v > m ? m : v;
}
// Per-axis type: 0 left-clipped, 1 interior, 2 right-clipped, 3 both (L = 1).
__host__ __device__ inline int ax_type(const Geo& g, int i) {
  if (g.L == 1) return 3;
  if (i == 0) return 0;
  if (i == g.L - 1) return 2;
  return 1;
}

// Owners of node column a (1 <= a <= Ln - 1) along a p = 1 box: subdomain i spans columns
// max(1, i n - delta + 1) .. min(Ln - 1, (i + 1) n + delta - 1), so the owners are
// i = ceil((a - delta + 1)/n) - 1 .. floor((a + delta - 1)/n) (clipped to 0 .. L - 1), one or two
// of them as 2 delta < n; returned as the owner table holds them: {first owner, its local
// column, second owner or -1, 0}.
__host__ __device__ inline int4 p1_owners(const Geo& g, int a) {
  const int u = a - g.delta + 1;
  const int ilo = u <= 0 ? 0 : (u + g.n - 1) / g.n - 1;
  const int hi = (a + g.delta - 1) / g.n;
  const int ihi = hi < g.L - 1 ? hi : g.L - 1;
  const int lo0 = ilo * g.n - g.delta + 1, lo1 = ihi * g.n - g.delta + 1;
  const int l0 = a - (lo0 > 1 ? lo0 : 1);
  return ihi > ilo ? make_int4(ilo, l0, ihi, a - (lo1 > 1 ? lo1 : 1)) : make_int4(ilo, l0, -1, 0);
}

// The float-pair stencil table holds each class's taps and one zero pad, so that a class's
// row is a whole number of aligned 16-byte loads: 9 + 1 (p = 1, five loads), 27 + 1 (p = 2,
// fourteen loads).
constexpr int kPairTapStride = 10;
constexpr int kPairTapStride3 = 28;
inline int pair_tap_stride(int p) { return p == 1 ? kPairTapStride : kPairTapStride3; }

// Subdomain descriptor on the device.
struct Sub {
  int type;     // compact type id
  int lo1, lo2; // first interior node column per axis (lo2 unused for p = 1)
  int w1, w2;   // widths in columns (w2 = 1 for p = 1)
  int nloc;     // w1 * w2 * nyi
};

// Scalars of the PCG iteration, resident on the device.
struct PcgState {
  double rho;      // (r, z) of the current z
  double pq;       // (p, A p)
  double alpha, beta;
  double rr;       // (r, r)
  double rr0;      // (r_0, r_0)
  double tol2;     // rtol^2 rr0
  double zq;       // (z_new, q) for the flexible variant
  int iter, maxit, done, status;
  int flexible;
  int pad_[3];
};

// Scalars of one SI-LOPCG Rayleigh-Ritz step (Algorithm 1): Gram matrices (upper triangles,
// entries (0,0) (0,1) (0,2) (1,1) (1,2) (2,2)) of S = [x_k, w_k, x_{k-1}] under A_sigma and M,
// the sums of the three vectors, the Ritz coefficients c and value theta (shifted by -sigma).
struct LopState {
  double GA[6], GB[6], sums[3];
  double c[3];
  double theta;
  double rr, mm, xmx;   // after the update: ||A_sigma x - theta M x||^2, ||M x||^2, x^T M x
  int m, status;
};

// Scalars of the outer iteration.
struct OuterState {
  double wMw, wsum, scale;
  double xAx;      // x^T A_sigma x
  double rr, mm;   // ||A_sigma x - mu M x||^2, ||M x||^2
  double lam_shift;
  int status;
  int pad_;
};

enum KernelClass {
  KC_STENCIL = 0, KC_PUPDATE, KC_XRUPDATE, KC_LOCAL_FP64, KC_PACK, KC_GEMM, KC_PROLONG,
  KC_CRESTRICT, KC_CSOLVE, KC_OUTER, KC_MISC, KC_RR, KC_PACK_XR, KC_COUNT
};

struct Timer {
  long long launches[KC_COUNT] = {};
  double ms[KC_COUNT] = {};
  std::vector<cudaEvent_t> pool;
  std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> pending;
};

}  // namespace dd

struct dd_ctx {
  dd_grid grid;
  dd::Geo g;
  cudaStream_t user_stream = nullptr;  // the caller's stream (may be the legacy NULL stream)
  cudaStream_t stream = nullptr;       // private non-blocking stream ordered after user_stream
  cudaStream_t side = nullptr;         // concurrent coarse branch
  cudaEvent_t ev_enter = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  int device = 0;
  int stage = 0;
  std::string err;
  long long bytes = 0;
  std::vector<void*> allocs;

  // options
  int check_every = 16;             // PCG iterations per graph replay between host checks
  int use_graph = 1;
  int flexible_opt = -1;
  int timing = 0;
  int fused_pq_opt = -1;            // p = 1: one kernel for p = z + beta p and q = A_sigma p (-1, 1) or two (0)
  int prolong_arith = 0;            // p = 1: prolong-sum owners in closed form (checked against the tables)
  int prolong_closed = 0;           // the closed form reproduces the tables
  int prolong_tables_opt = 1;       // 0: owners in closed form where it holds (slower: 28.1 against 24.5 us at L = 2048)
  int4 ptypes = {0, 0, 0, 0};       // p = 1: type ids of the left end, interior and right end subdomains
  int pdl = 0;                      // PCG chain kernels launched with programmatic dependent launch
  int fuse_xr_opt = 0;              // x/r update fused into the packing: 1 on, 0 or -1 off
  int matvec_tiled = 1;             // p = 2 float pairs: the shared-memory tiled matvec where it fits
  // x_{k+1} = x_k + alpha_k p_k deferred to iteration k + 1's p update, which reads p_k anyway,
  // and one final update after the last iteration: the x/r update then streams r and q only
  int x_lag = 1;
  int fuse_xr = 0;                  // the resolved choice
  int pq_pairs_opt = -1;            // q = A_sigma p of the fused p = 1 kernel: -1 automatic, 0 FP64, 1 float pairs
  int pq_pairs = 0;                 // the resolved choice
  dd::Timer timer;

  // types and subdomains
  int ntypes = 0;
  int type_ax[dd::kMaxTypes][2];   // per-axis types of each compact type
  int type_nloc[dd::kMaxTypes];
  int type_w1[dd::kMaxTypes], type_w2[dd::kMaxTypes];
  std::vector<dd::Sub> subs_h;
  std::vector<int> type_count;      // subdomains per type
  std::vector<int> type_first;      // first slot (subdomains sorted by type)
  dd::Sub* subs = nullptr;          // device, indexed by subdomain id
  int4* axown = nullptr;            // device, per x node column a: {owner0, local col0, owner1 or -1, local col1}
  int4* subrow = nullptr;           // device, per subdomain: {row offset in Y (slot kpad), type kpad, w2, nloc}
  int* slot_of_sub = nullptr;       // device: subdomain id -> packed row (type-sorted)
  int* sub_of_slot = nullptr;       // device: packed row -> subdomain id
  int2* groups = nullptr;           // device: {first slot, count} of same-type slots solved by one warp
  int ngroups = 0, rhs_k = 1;       // FP64 local solves: groups and right-hand sides per warp
  std::vector<int2> group_h;        // host copy of groups
  int nloc_max = 0, kpad = 0, band = 0;

  // V and stencil tables [tap][cls]
  double* Vqp = nullptr;
  double* tabA = nullptr;   // K + M_V
  double* tabM = nullptr;   // M
  double* tabS = nullptr;   // K + M_V - sigma M
  float2* tabS2 = nullptr;  // tabS as float pairs (hi, lo), class-major [cls][pair_tap_stride(p)]
  float2* p2 = nullptr;     // p = 2: the current PCG direction as float pairs (guard band as the vectors)
  int4* colrow = nullptr;   // p = 1: per node column, each owner's packed-row and type-row offsets there
  double* tabL = nullptr;   // K + M_V - lambda M (adjoint of the eigenvector)
  double* qp_part = nullptr;      // quadrature-point reduction partials
  long long qp_part_len = 0;
  double* gv[8] = {};             // gradient work vectors
  double* gscal = nullptr;        // device scalars of the gradient projections
  // GMRES (restart gm_restart): basis V[0..m], preconditioned directions Z[0..m-1]
  int krylov = 0;                 // inner solver of the eigen-iterations: 0 PCG, 1 GMRES
  int gm_restart = 30, gm_alloc = 0;
  std::vector<double*> gm_V, gm_Z;
  double* gm_W = nullptr;
  double** gm_Vptr = nullptr;
  double** gm_Zptr = nullptr;
  double *gm_part = nullptr, *gm_h = nullptr, *gm_H = nullptr, *gm_cs = nullptr, *gm_sn = nullptr;
  double *gm_g = nullptr, *gm_y = nullptr, *gm_res = nullptr, *gm_res_h = nullptr;
  double* gout = nullptr;         // gradient staging (n_V doubles)

  // cell problem
  long long ncell = 0;
  int cell_band = 0;
  double sigma = 0.0;
  int cell_iters = 0;
  double* psi_cell = nullptr;      // natural cell order
  double* wT = nullptr;            // coarse weights per type [type][kpad]: D_i R_i psi
  double* puT = nullptr;           // partition of unity per type [type][kpad]: D_i
  float* wT32 = nullptr;           // FP32 copies of wT and puT (the prolong-sum of the mixed form)
  float* puT32 = nullptr;
  int ras = 0;                     // 1: restricted local prolongation (M_RAS2^{-1})
  int gemm_bn_opt = 0;             // local-solve GEMM N tile: 0 autotuned, 128, 160 or 256
  float* ysc = nullptr;            // FP8: per packed row 1 / (s_i s_T) (undoes the operand scales)
  float* ascale = nullptr;         // FP8: per type 1 / s_T
  double* ascale64 = nullptr;      // FP8: per type s_T = 448 / max|A_T^{-1}|
  int gemm_bn = 0;                 // the N tile chosen by the autotuner (or forced) at set-up

  // vectors (padded length plen)
  double *x = nullptr, *r = nullptr, *z = nullptr, *q = nullptr;
  double* pb[2] = {nullptr, nullptr};  // search directions: iteration k reads pb[k & 1], writes pb[(k + 1) & 1]
  double *w1 = nullptr, *w2 = nullptr, *w3 = nullptr;   // outer-iteration work vectors
  double* xe = nullptr;                                  // eigenvector iterate
  double *stage_a = nullptr, *stage_b = nullptr;         // unpadded staging (ndof)

  // local solves
  double* bandCB = nullptr;   // [type][nloc_max][band+1] column band of L
  double* bandRB = nullptr;   // [type][nloc_max][band+1] row band of L
  double* bandInv = nullptr;  // [type][nloc_max] 1/L_ii
  float* bandCB32 = nullptr;  // the same in FP32: the mixed form, whose inverses are rounded
  float* bandRB32 = nullptr;
  float* bandInv32 = nullptr;
  double* Y64 = nullptr;      // [nsub][kpad] local solutions (FP64 path)
  float* Y32 = nullptr;       // [nsub][kpad] local solutions (GEMM path)
  void* Ainv = nullptr;       // [type][kpad][kpad] rounded local inverses
  void* Rpack = nullptr;      // [nsub (type-sorted)][kpad] rounded restrictions
  void* tmapA = nullptr;      // CUtensorMap (host copy, 128 B)
  void* tmapB = nullptr;
  int gemm_ok = 0;
  int* dev_err = nullptr;     // device error word for bounded waits

  // coarse
  double* A0band = nullptr;   // p=1: [3][N] (sub, diag, super); p=2: [N][9]
  double* cr = nullptr;       // p=1 cyclic-reduction coefficients
  int cr_m = 0, cr_c2 = 0, cr_w2 = 0;   // cyclic reduction: levels + 1, packed multipliers, row arrays
  double* A0inv = nullptr;    // dense inverse [N][N] (p = 2; p = 1 on request)
  int coarse_mode = 0;        // 0 automatic, 1 cyclic reduction (p = 1), 2 dense inverse
  double *cf_CB = nullptr, *cf_RB = nullptr, *cf_inv = nullptr;   // banded factor of A_0
  int coarse_dense = 0;       // the form in use
  double* c0 = nullptr;       // coarse rhs [N]
  double* u0 = nullptr;       // coarse solution [N]
  float* u0f = nullptr;       // the same rounded to FP32 (mixed form)

  // reductions
  double* red = nullptr;      // partials
  unsigned* cnt = nullptr;    // last-block counters [16]
  dd::PcgState* st = nullptr;
  dd::OuterState* ost = nullptr;
  dd::PcgState* st_h = nullptr;    // pinned mirror
  dd::OuterState* ost_h = nullptr; // pinned mirror
  dd::LopState* lst = nullptr;     // SI-LOPCG step scalars (device)
  dd::LopState* lst_h = nullptr;   // pinned mirror
  double* lop_red = nullptr;       // partials of the 15 Gram sums
  double* lop[12] = {};            // SI-LOPCG work vectors (padded layout)

  // graph of one block of PCG iterations
  cudaGraphExec_t graph = nullptr;
  int graph_iters = 0;
  long long graph_kernels = 0;   // kernel nodes in one replay of the graph
};

// the x that the PCG p update advances (x_lag), or null when the x/r update does it
inline double* x_lag_target(dd_ctx* c) { return c->x_lag ? c->x : nullptr; }

namespace dd {

// One problem of a batched launch: its geometry, the device buffers of its context, and the
// block counts of its own plain launches (each batched kernel gives every block of problem i
// the index and count it has in problem i's plain launch, so that the arithmetic, and the
// order of every reduction, is that of the plain launch).
struct BInst {
  Geo g;
  double *x, *r, *z, *pb0, *pb1, *q, *w1, *w2, *w3, *xe;   // padded vectors
  const double *tabS, *tabM;
  const float2* tabS2;
  int pq_pairs;
  PcgState* st;
  OuterState* ost;
  double* red;
  unsigned* cnt;
  const Sub* subs;
  const int* slot_of_sub;
  void* Rpack;            // this problem's rows of the batch's packed restrictions
  const double* wT;
  double* c0;
  double* u0;
  float* u0f;
  const float* Y32;       // this problem's rows of the batch's local solutions
  const float* wT32;
  const float* puT32;
  const int4* axown;
  const int4* subrow;
  const int4* colrow;
  const double* cr;       // cyclic-reduction coefficients of A_0 (p = 1)
  int cr_m, cr_c2, cr_w2, cr_staged;
  int kpad, coarse, nsub, flexible;
  int nb_init, nb_fused, nb_xr, nb_prolong, nb_sdot, nb_st, nb_vec, nb_st2;
  int active;             // 0 once the problem's eigen-iteration has stopped
  int* err;               // the context's error word of bounded waits
  double* lop[12];        // SI-LOPCG work vectors (padded)
  LopState* lst;
  double* lop_red;
  int4 ptypes;            // p = 1: type ids of the left end, interior and right end subdomains
  int prolong_arith;      // the prolong-sum's owners computed in closed form (p = 1)
};

// Vector roles in BInst (the batched outer-step kernels take roles, not pointers);
// BV_LOP + k is the SI-LOPCG work vector lop[k].
enum BVec { BV_X = 0, BV_R, BV_Z, BV_Q, BV_W1, BV_W2, BV_W3, BV_XE, BV_NONE = 15, BV_LOP = 16 };

// Per-problem scalars copied to the host after a batched step.
struct BStat {
  int pcg_done, pcg_status, pcg_iter, active;
  double xAx, rr, mm;
  int outer_status, lop_status;
  double theta, lop_rr, lop_mm;
};

// ----- launchers (kernels in k_*.cu) -----
int grid_blocks(long long work, int threads, int max_per_sm = 8);

void launch_build_tables(dd_ctx* c);
void launch_tabS(dd_ctx* c, double sigma);
void launch_stencil(dd_ctx* c, const double* tab, const double* x, double* y, cudaStream_t s);
void launch_stencil_dot(dd_ctx* c, const double* tab, const double* x, double* y, double* out_dot,
                        unsigned* counter, cudaStream_t s);
void launch_pad(dd_ctx* c, const double* u, double* v, cudaStream_t s);     // unpadded -> padded
void launch_unpad(dd_ctx* c, const double* v, double* u, cudaStream_t s);   // padded -> unpadded
void launch_check_finite(const double* v, long long n, int* flag, cudaStream_t s);

// PCG pieces
void launch_pcg_init(dd_ctx* c, const double* b, cudaStream_t s);   // r = b - A x, rr0
void launch_pupdate(dd_ctx* c, cudaStream_t s);                     // p = z + beta p
void launch_matvec_pq(dd_ctx* c, cudaStream_t s);                   // q = A p, pq, alpha
void launch_pupdate_pairs(dd_ctx* c, cudaStream_t s);               // p = 2: p update, p also as float pairs
void launch_matvec_pq_pairs(dd_ctx* c, cudaStream_t s);             // p = 2: q = A p in float pairs, pq, alpha
void launch_fused_pq(dd_ctx* c, cudaStream_t s);                    // p = z + beta p; q = A p; pq (p = 1)
void launch_xr_update(dd_ctx* c, cudaStream_t s);                   // x (unless x_lag), r, rr, done
void launch_x_final(dd_ctx* c, cudaStream_t s);                      // x_lag: the last x += alpha p
// z = ..., rz, beta; upd (iterations): r -= alpha q first, the x update having run in launch_pack_xr
void launch_prolong(dd_ctx* c, int init, cudaStream_t s, double* zout = nullptr, bool upd = false);
void launch_precond(dd_ctx* c, const double* r, double* z, int pcg_mode, cudaStream_t s);

// local solves
template <typename T>
void launch_local_assemble(dd_ctx* c, T* CB);
// banded Cholesky of nmat matrices (orders in sizes_host, or all n when null); T double or float
template <typename T>
int launch_band_factor(dd_ctx* c, T* CB, T* RB, T* inv, int nmat, int n, int b, int* flag, const int* sizes_host);
void launch_band_solve_local(dd_ctx* c, const double* r, double* c0, cudaStream_t s);
template <typename T>
void launch_band_inverse_rows(int n, int b, const T* CB, const T* RB, const T* inv, T* out, cudaStream_t s);

// cell problem
int cell_eigenpair(dd_ctx* c);

// coarse
void launch_coarse_weights(dd_ctx* c);
int coarse_assemble(dd_ctx* c, cudaStream_t s);
int coarse_factor(dd_ctx* c);
void launch_coarse_restrict(dd_ctx* c, const double* r, cudaStream_t s);
void launch_coarse_solve(dd_ctx* c, cudaStream_t s);

// GEMM path
int gemm_setup(dd_ctx* c);
void launch_pack(dd_ctx* c, const double* r, double* c0, cudaStream_t s);
void launch_pack_xr(dd_ctx* c, cudaStream_t s);   // p = 1 iteration: x update, (r, r), stop test and the packing
int launch_gemm(dd_ctx* c, cudaStream_t s);
void gemm_free(dd_ctx* c);

// outer iteration
void launch_outer_normalize(dd_ctx* c, const double* w, double* Mw, double* xout, cudaStream_t s);
void launch_outer_residual(dd_ctx* c, const double* xe, const double* Mx, double* Ax, cudaStream_t s,
                           double* ro = nullptr);
void launch_outer_dots(dd_ctx* c, const double* w, const double* Mw, cudaStream_t s);
void launch_lop_gram(dd_ctx* c, const double* const S[3], const double* const AS[3], const double* const MS[3],
                     double drop, cudaStream_t s);
void launch_lop_update(dd_ctx* c, const double* x, const double* w, const double* xp, double* out,
                       cudaStream_t s);
void launch_lop_normalize(dd_ctx* c, double* x, double* Mx, cudaStream_t s);
void launch_lop_update3(dd_ctx* c, const double* const S[3], const double* const AS[3], const double* const MS[3],
                        double* x, double* Ax, double* Mx, double* ro, cudaStream_t s);
void launch_stencil2(dd_ctx* c, const double* tab1, const double* tab2, const double* x, double* y1, double* y2,
                     cudaStream_t s);
void launch_set_entry(double* v, long long idx, double val, cudaStream_t s);
void launch_qp_product(dd_ctx* c, const double* u, const double* v, double* out, cudaStream_t s);
void launch_dot(dd_ctx* c, const double* a, const double* b, double* out, cudaStream_t s);
void launch_axpby(dd_ctx* c, double ca, const double* x, double cb_scale, const double* cb, const double* y,
                  double* out, cudaStream_t s);
void launch_tab_shift(dd_ctx* c, double shift, double* dst);
void launch_multidot(dd_ctx* c, int nv, const double* const* V, const double* w, double* h, int accumulate,
                     cudaStream_t s);
void launch_multiaxpy(dd_ctx* c, int nv, const double* const* V, const double* coef, double sign, double* w,
                      cudaStream_t s);
void launch_scale_by_norm(dd_ctx* c, const double* w, const double* nrm2, double* v, cudaStream_t s);
void launch_givens(dd_ctx* c, int j, cudaStream_t s);
void launch_backsolve(dd_ctx* c, int m, cudaStream_t s);
void launch_gmres_start(dd_ctx* c, const double* nrm2, cudaStream_t s);
void launch_add_inplace(dd_ctx* c, int n, double* a, const double* b, cudaStream_t s);

// ----- batched launchers (vmap[k] = {problem, block within the problem's launch}) -----
void batch_grid_sizes(const dd_ctx* c, BInst* I);   // the nb_* of the plain launchers
void launch_b_pcg_reset(const BInst* B, int n, double rtol2, int maxit, cudaStream_t s);
void launch_b_zero_pcg(const BInst* B, const int2* vmap, int nvb, cudaStream_t s);
void launch_b_pcg_init(const BInst* B, const int2* vmap, int nvb, int b_role, cudaStream_t s);
void launch_b_fused_pq(const BInst* B, const int2* vmap, int nvb, int ypad, bool pairs, cudaStream_t s);
void launch_b_xr_update(const BInst* B, const int2* vmap, int nvb, cudaStream_t s);
void launch_b_prolong(const BInst* B, const int2* vmap, int nvb, int mode, bool arith, bool upd, cudaStream_t s);
void launch_b_pack_xr(const BInst* B, const int2* vmap, int nvb, int precision, cudaStream_t s);
void launch_b_stencil(const BInst* B, const int2* vmap, int nvb, int mass, int x_role, int y_role, cudaStream_t s);
void launch_b_stencil_dot(const BInst* B, const int2* vmap, int nvb, int x_role, int y_role, cudaStream_t s);
void launch_b_outer_normalize(const BInst* B, const int2* vmap, int nvb, int w_role, int mw_role, int x_role,
                              cudaStream_t s);
void launch_b_outer_res(const BInst* B, const int2* vmap, int nvb, int ax_role, int mx_role, cudaStream_t s);
void launch_b_gather(const BInst* B, int n, BStat* out, cudaStream_t s);
void launch_b_mark_done(const BInst* B, int n, cudaStream_t s);
void launch_b_pack(const BInst* B, const int2* vmap, int nvb, int precision, cudaStream_t s);
void launch_b_cr_solve(const BInst* B, int n, size_t smem, cudaStream_t s);
void cr_launch_shape(const dd_ctx* c, size_t* smem, int* staged);
struct BGemm;   // grouped local-solve contraction of a batch (k_gemm.cu)
BGemm* bgemm_create(const std::vector<dd_ctx*>& cs, const std::vector<int>& type_base,
                    const std::vector<int>& slot_base, void* Ainv_all, void* Rpack_all, float* Y_all, int* err,
                    cudaStream_t s);
void bgemm_run(BGemm* b, int bn, cudaStream_t s);
int bgemm_tune(BGemm* b, cudaStream_t s);
void bgemm_destroy(BGemm* b);
void launch_b_unpad(const BInst* B, const int2* vmap, int nvb, int src_role, double* const* dst, cudaStream_t s);
// (active problems only)
void launch_b_pad(const BInst* B, const int2* vmap, int nvb, const double* const* src, int dst_role, cudaStream_t s);
void launch_b_zero_roles(const BInst* B, const int2* vmap, int nvb, int first_role, int nroles, cudaStream_t s);
void launch_b_set_entry(const BInst* B, int n, int role, long long idx, double val, cudaStream_t s);
void launch_b_stencil_role(const BInst* B, const int2* vmap, int nvb, int mass, int x_role, int y_role,
                           cudaStream_t s);
void launch_b_stencil2(const BInst* B, const int2* vmap_st2, int nvb, int x_role, int ys_role, int ym_role,
                       cudaStream_t s);
void launch_b_lop_normalize(const BInst* B, const int2* vmap, int nvb, int x_role, int mx_role, cudaStream_t s);
void launch_b_outer_res_ro(const BInst* B, const int2* vmap, int nvb, int ax_role, int mx_role, int ro_role,
                           cudaStream_t s);
void launch_b_lop_gram(const BInst* B, const int2* vmap, int nvb, const int* S, const int* AS, const int* MS,
                       double drop, cudaStream_t s);
void launch_b_lop_update3(const BInst* B, const int2* vmap, int nvb, const int* S, const int* AS, const int* MS,
                          int x_role, int ax_role, int mx_role, int ro_role, cudaStream_t s);
void launch_b_lop_reset(const BInst* B, int n, cudaStream_t s);
void launch_b_unpad_active(const BInst* B, const int2* vmap, int nvb, int src_role, double* const* dst,
                           cudaStream_t s);
constexpr int kMaxRedBlocksHost = 4096;   // partial slots per reduced value (kMaxRedBlocks)
void launch_b_outer_dots_roles(const BInst* B, const int2* vmap, int nvb, int w_role, int mw_role, cudaStream_t s);
double* alloc_vec(dd_ctx* c);


// timing helpers
void timer_begin(dd_ctx* c, int kc, cudaStream_t s, cudaEvent_t* e0);
void timer_end(dd_ctx* c, int kc, cudaStream_t s, cudaEvent_t e0);
void timer_collect(dd_ctx* c);

void* dev_alloc(dd_ctx* c, size_t bytes);
void launch_fill(double* x, long long n, double v, cudaStream_t s);

// process-wide count of kernel launches issued by this library (graph replays included)
void note_launch();
void note_launches(long long k);
long long launch_count();
void set_capturing(bool on);                  // this thread is capturing a graph
long long graph_kernel_nodes(cudaGraph_t gr);

}  // namespace dd

#define DD_CUDA(call)                                                          \
  do {                                                                         \
    cudaError_t e_ = (call);                                                   \
    if (e_ != cudaSuccess) {                                                   \
      throw dd::Error(DD_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    }                                                                          \
  } while (0)

namespace dd {
struct Error {
  int code;
  std::string msg;
  Error(int c, std::string m) : code(c), msg(std::move(m)) {}
};
}  // namespace dd

#include <atomic>
#include <utility>

namespace dd {
// Launch of a kernel of the PCG iteration's chain.  With pdl set, the launch carries the
// programmatic-serialization attribute: the kernel's blocks may be scheduled while its
// predecessor on the stream drains, and wait in griddepcontrol.wait (pdl_wait) until the
// predecessor has completed and its writes are visible.  Without it, a plain launch.
template <typename... KArgs, typename... Args>
void launch_chain(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s, bool pdl,
                  Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = pdl ? at : nullptr;
  cfg.numAttrs = pdl ? 1 : 0;
  DD_CUDA(cudaLaunchKernelEx(&cfg, kern, std::forward<Args>(args)...));
  note_launch();
}
}  // namespace dd

namespace dd {
// cudaFuncSetAttribute (dynamic shared-memory opt-in) applies to the current device only, so
// a "set once" flag must remember every device ordinal it has been set on.  Ordinals up to 63
// are remembered in one word; higher ordinals set the attribute on every call.
struct PerDeviceOnce {
  std::atomic<unsigned long long> done{0};
};
template <typename F>
inline void once_per_device(PerDeviceOnce& o, F&& f) {
  int dev = 0;
  DD_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) {
    f();
    return;
  }
  const unsigned long long bit = 1ull << dev;
  if (o.done.load(std::memory_order_acquire) & bit) return;
  f();   // idempotent: two threads racing here both set the same attribute
  o.done.fetch_or(bit, std::memory_order_release);
}
}  // namespace dd
