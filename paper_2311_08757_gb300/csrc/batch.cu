// Batched ground states: many independent instances (uneven L, own potential and shift).
//
// Set-up (cell eigenpair, local inverses, coarse matrix) runs per instance, each on its own
// context and private stream, on a pool of host threads (largest instance first), so that
// the instances' set-up kernels overlap on the GPU; its cost does not grow with L.
//
// The inverse iteration then runs batched when the instances share everything but L, the
// potential and the shift (p = 1, rounded local inverses, same h, delta, ell, quadrature and
// partition of unity): every kernel of a PCG iteration is ONE launch over all instances --
// its blocks are the blocks of every instance's own launch (block index and count within
// the instance), the local-solve contraction is one grouped tensor-core launch over all
// instances' tiles -- and a block of iterations of all instances is one CUDA graph.  Each
// instance keeps its own device scalars (PCG state, outer state); kernels of an instance
// whose solve is done return at once, and an instance whose eigen-iteration has stopped
// drops out of every launch.  The outer steps run in lockstep; results equal those of the
// single-instance calls bit for bit.  Other combinations (p = 2, the plain FP64 form, SI-
// LOPCG) run as concurrent per-instance pipelines.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstring>
#include <limits>
#include <mutex>
#include <thread>
#include <vector>

#include "dd_internal.h"

struct dd_batch {
  std::vector<dd_ctx*> ctx;
  std::vector<double*> x;      // per instance: device start vector / solution (ndof)
  std::vector<long long> ndof;
  int device = 0;
  std::string err;

  // batched engine
  bool eligible = false;
  int precision = 0;
  void* Ainv_all = nullptr;    // [sum of types][kpad][kpad] rounded local inverses
  void* Rpack_all = nullptr;   // [sum of subdomains][kpad] packed restrictions
  float* Y_all = nullptr;      // [sum of subdomains][kpad] local solutions
  std::vector<int> type_base, slot_base;
  std::vector<dd::BInst> Bh;
  dd::BInst* B = nullptr;
  int2 *vm_init = nullptr, *vm_fused = nullptr, *vm_xr = nullptr, *vm_prolong = nullptr, *vm_sdot = nullptr,
       *vm_st = nullptr, *vm_vec = nullptr, *vm_pack = nullptr, *vm_st2 = nullptr;
  int n_init = 0, n_fused = 0, n_xr = 0, n_prolong = 0, n_sdot = 0, n_st = 0, n_vec = 0, n_pack = 0, n_st2 = 0;
  size_t cr_smem = 0;
  int ypad = 0;
  dd::BGemm* gemm = nullptr;
  int bn = 0;                  // N tile of the grouped contraction (autotuned)
  int check_every = 8;         // PCG iterations per graph replay
  cudaStream_t s = nullptr, side = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  cudaGraphExec_t graph = nullptr;
  long long graph_kernels = 0;
  dd::BStat* stat_d = nullptr;
  dd::BStat* stat_h = nullptr;
  double** xptr_d = nullptr;   // device array of the instances' start / solution vectors
  int* err_d = nullptr;        // error word of the grouped contraction's bounded waits
  bool built = false;
  int last_batched = 0;        // the last dd_batch_ground_states ran the batched kernels
};

namespace {

using dd::BInst;
using dd::BStat;

__global__ void k_fill(long long n, double v, double* x) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n;
       t += (long long)gridDim.x * blockDim.x)
    x[t] = v;
}

void free_engine(dd_batch* b) {
  if (b->graph) cudaGraphExecDestroy(b->graph);
  b->graph = nullptr;
  dd::bgemm_destroy(b->gemm);
  b->gemm = nullptr;
  for (void* p : {(void*)b->B, (void*)b->vm_init, (void*)b->vm_fused, (void*)b->vm_xr, (void*)b->vm_prolong,
                  (void*)b->vm_sdot, (void*)b->vm_st, (void*)b->vm_vec, (void*)b->vm_pack, (void*)b->stat_d,
                  (void*)b->xptr_d, (void*)b->err_d, (void*)b->vm_st2})
    if (p) cudaFree(p);
  b->B = nullptr;
  b->vm_init = b->vm_fused = b->vm_xr = b->vm_prolong = b->vm_sdot = b->vm_st = b->vm_vec = b->vm_pack = nullptr;
  b->vm_st2 = nullptr;
  b->stat_d = nullptr;
  b->xptr_d = nullptr;
  b->err_d = nullptr;
  if (b->stat_h) cudaFreeHost(b->stat_h);
  b->stat_h = nullptr;
  if (b->side) cudaStreamDestroy(b->side);
  if (b->s) cudaStreamDestroy(b->s);
  if (b->ev_fork) cudaEventDestroy(b->ev_fork);
  if (b->ev_join) cudaEventDestroy(b->ev_join);
  b->side = b->s = nullptr;
  b->ev_fork = b->ev_join = nullptr;
  b->built = false;
}

void destroy_all(dd_batch* b) {
  free_engine(b);
  for (double* p : b->x)
    if (p) cudaFree(p);
  for (dd_ctx* c : b->ctx) dd_destroy(c);
  for (void* p : {b->Ainv_all, b->Rpack_all, (void*)b->Y_all})
    if (p) cudaFree(p);
  delete b;
}

// the instances share everything the batched kernels and the grouped contraction need
bool batchable(const dd_batch* b) {
  const dd_ctx* c0 = b->ctx.front();
  const dd_grid& g0 = c0->grid;
  if (g0.p != 1 || g0.coarse != 1) return false;
  if (g0.precision != DD_PREC_BF16 && g0.precision != DD_PREC_TF32) return false;
  for (const dd_ctx* c : b->ctx) {
    const dd_grid& g = c->grid;
    if (g.p != g0.p || g.n != g0.n || g.overlap != g0.overlap || g.quad_pts != g0.quad_pts ||
        g.pu_kind != g0.pu_kind || g.precision != g0.precision || g.coarse != g0.coarse ||
        c->g.ny != c0->g.ny || c->g.Ypad != c0->g.Ypad || c->kpad != c0->kpad)
      return false;
  }
  return true;
}

int2* upload_vmap(const std::vector<int2>& v) {
  int2* d = nullptr;
  DD_CUDA(cudaMalloc(&d, sizeof(int2) * std::max<size_t>(1, v.size())));
  DD_CUDA(cudaMemcpy(d, v.data(), sizeof(int2) * v.size(), cudaMemcpyHostToDevice));
  return d;
}

// descriptors, block maps, streams, the grouped contraction (after every coarse build)
void build_engine(dd_batch* b) {
  const int n = (int)b->ctx.size();
  DD_CUDA(cudaSetDevice(b->device));
  DD_CUDA(cudaStreamCreateWithFlags(&b->s, cudaStreamNonBlocking));
  DD_CUDA(cudaStreamCreateWithFlags(&b->side, cudaStreamNonBlocking));
  DD_CUDA(cudaEventCreateWithFlags(&b->ev_fork, cudaEventDisableTiming));
  DD_CUDA(cudaEventCreateWithFlags(&b->ev_join, cudaEventDisableTiming));
  DD_CUDA(cudaMalloc(&b->err_d, sizeof(int) * 16));
  DD_CUDA(cudaMemset(b->err_d, 0, sizeof(int) * 16));
  b->Bh.assign(n, BInst());
  std::vector<int2> vinit, vfused, vxr, vprol, vsdot, vst, vst2, vvec, vpack;
  b->cr_smem = 0;
  for (int i = 0; i < n; ++i) {
    dd_ctx* c = b->ctx[i];
    BInst& I = b->Bh[i];
    std::memset(&I, 0, sizeof(I));
    I.g = c->g;
    I.x = c->x; I.r = c->r; I.z = c->z; I.pb0 = c->pb[0]; I.pb1 = c->pb[1]; I.q = c->q;
    I.w1 = c->w1; I.w2 = c->w2; I.w3 = c->w3; I.xe = c->xe;
    I.tabS = c->tabS; I.tabM = c->tabM;
    I.st = c->st; I.ost = c->ost; I.red = c->red; I.cnt = c->cnt;
    I.subs = c->subs; I.slot_of_sub = c->slot_of_sub; I.Rpack = c->Rpack; I.wT = c->wT; I.c0 = c->c0;
    I.u0 = c->u0; I.u0f = c->u0f; I.Y32 = c->Y32; I.wT32 = c->wT32; I.puT32 = c->puT32;
    I.axown = c->axown; I.subrow = c->subrow; I.cr = c->cr;
    I.cr_m = c->cr_m; I.cr_c2 = c->cr_c2; I.cr_w2 = c->cr_w2;
    size_t smem = 0;
    int staged = 0;
    dd::cr_launch_shape(c, &smem, &staged);
    I.cr_staged = staged;
    b->cr_smem = std::max(b->cr_smem, smem);
    I.kpad = c->kpad; I.coarse = 1; I.nsub = c->g.nsub;
    I.flexible = (c->flexible_opt < 0) ? 1 : c->flexible_opt;
    I.err = c->dev_err;
    I.active = 1;
    dd::batch_grid_sizes(c, &I);
    for (int k = 0; k < I.nb_init; ++k) vinit.push_back(make_int2(i, k));
    for (int k = 0; k < I.nb_fused; ++k) vfused.push_back(make_int2(i, k));
    for (int k = 0; k < I.nb_xr; ++k) vxr.push_back(make_int2(i, k));
    for (int k = 0; k < I.nb_prolong; ++k) vprol.push_back(make_int2(i, k));
    for (int k = 0; k < I.nb_sdot; ++k) vsdot.push_back(make_int2(i, k));
    for (int k = 0; k < I.nb_st; ++k) vst.push_back(make_int2(i, k));
    for (int k = 0; k < I.nb_st2; ++k) vst2.push_back(make_int2(i, k));
    for (int k = 0; k < I.nb_vec; ++k) vvec.push_back(make_int2(i, k));
    for (int k = 0; k < c->g.nsub; ++k) vpack.push_back(make_int2(i, k));
  }
  if (b->cr_smem > 220 * 1024) throw dd::Error(DD_EINVAL, "coarse chain too long for the batched cyclic reduction");
  b->ypad = b->ctx.front()->g.Ypad;
  b->vm_init = upload_vmap(vinit); b->n_init = (int)vinit.size();
  b->vm_fused = upload_vmap(vfused); b->n_fused = (int)vfused.size();
  b->vm_xr = upload_vmap(vxr); b->n_xr = (int)vxr.size();
  b->vm_prolong = upload_vmap(vprol); b->n_prolong = (int)vprol.size();
  b->vm_sdot = upload_vmap(vsdot); b->n_sdot = (int)vsdot.size();
  b->vm_st = upload_vmap(vst); b->n_st = (int)vst.size();
  b->vm_st2 = upload_vmap(vst2); b->n_st2 = (int)vst2.size();
  b->vm_vec = upload_vmap(vvec); b->n_vec = (int)vvec.size();
  b->vm_pack = upload_vmap(vpack); b->n_pack = (int)vpack.size();
  DD_CUDA(cudaMalloc(&b->B, sizeof(BInst) * n));
  DD_CUDA(cudaMemcpy(b->B, b->Bh.data(), sizeof(BInst) * n, cudaMemcpyHostToDevice));
  DD_CUDA(cudaMalloc(&b->stat_d, sizeof(BStat) * n));
  DD_CUDA(cudaMallocHost(&b->stat_h, sizeof(BStat) * n));
  DD_CUDA(cudaMalloc(&b->xptr_d, sizeof(double*) * n));
  DD_CUDA(cudaMemcpy(b->xptr_d, b->x.data(), sizeof(double*) * n, cudaMemcpyHostToDevice));
  b->gemm = dd::bgemm_create(b->ctx, b->type_base, b->slot_base, b->Ainv_all, b->Rpack_all, b->Y_all, b->err_d + 8,
                             b->s);
  // autotune the grouped contraction's N tile on the batch's operands (done flags cleared)
  dd::launch_b_pcg_reset(b->B, n, 1.0, 1, b->s);
  b->bn = dd::bgemm_tune(b->gemm, b->s);
  DD_CUDA(cudaStreamSynchronize(b->s));
  b->built = true;
}

void upload_active(dd_batch* b) {
  DD_CUDA(cudaMemcpyAsync(b->B, b->Bh.data(), sizeof(BInst) * b->Bh.size(), cudaMemcpyHostToDevice, b->s));
}

// z = M_AS2^{-1} r for every active instance (mode 1: PCG start, 2: iteration); the coarse
// solves run on the side stream beside the grouped contraction (the operator is additive)
void precond(dd_batch* b, int mode) {
  dd::launch_b_pack(b->B, b->vm_pack, b->n_pack, b->precision, b->s);
  DD_CUDA(cudaEventRecord(b->ev_fork, b->s));
  DD_CUDA(cudaStreamWaitEvent(b->side, b->ev_fork, 0));
  dd::launch_b_cr_solve(b->B, (int)b->ctx.size(), b->cr_smem, b->side);
  DD_CUDA(cudaEventRecord(b->ev_join, b->side));
  dd::bgemm_run(b->gemm, b->bn, b->s);
  DD_CUDA(cudaStreamWaitEvent(b->s, b->ev_join, 0));
  dd::launch_b_prolong(b->B, b->vm_prolong, b->n_prolong, mode, b->s);
}

void pcg_iteration(dd_batch* b) {
  dd::launch_b_fused_pq(b->B, b->vm_fused, b->n_fused, b->ypad, b->s);
  dd::launch_b_xr_update(b->B, b->vm_xr, b->n_xr, b->s);
  precond(b, 2);
}

void build_graph(dd_batch* b) {
  if (b->graph) {
    cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
  }
  cudaGraph_t gr;
  const long long before = dd::launch_count();
  DD_CUDA(cudaStreamBeginCapture(b->s, cudaStreamCaptureModeThreadLocal));
  try {
    for (int i = 0; i < b->check_every; ++i) pcg_iteration(b);
  } catch (...) {
    cudaStreamEndCapture(b->s, &gr);
    cudaGetLastError();
    dd::note_launches(before - dd::launch_count());
    throw;
  }
  DD_CUDA(cudaStreamEndCapture(b->s, &gr));
  b->graph_kernels = dd::launch_count() - before;
  dd::note_launches(-b->graph_kernels);   // replays are counted when launched
  DD_CUDA(cudaGraphInstantiate(&b->graph, gr, 0));
  DD_CUDA(cudaGraphDestroy(gr));
}

void gather(dd_batch* b) {
  const int n = (int)b->ctx.size();
  dd::launch_b_gather(b->B, n, b->stat_d, b->s);
  DD_CUDA(cudaMemcpyAsync(b->stat_h, b->stat_d, sizeof(BStat) * n, cudaMemcpyDeviceToHost, b->s));
  DD_CUDA(cudaStreamSynchronize(b->s));
}

// b = M x_k (w2) -> x_{k+1} = w / ||w||_M (xe), A_sigma x and the residual norms; as the
// plain outer step
void outer_images(dd_batch* b, int w_role) {
  dd::launch_b_stencil(b->B, b->vm_st, b->n_st, 1, w_role, dd::BV_W2, b->s);
  dd::launch_b_outer_normalize(b->B, b->vm_vec, b->n_vec, w_role, dd::BV_W2, dd::BV_XE, b->s);
  dd::launch_b_stencil_dot(b->B, b->vm_sdot, b->n_sdot, dd::BV_XE, dd::BV_W3, b->s);
  dd::launch_b_outer_res(b->B, b->vm_vec, b->n_vec, dd::BV_W3, dd::BV_W2, b->s);
}

// Batched shifted inverse iteration (the stop rule and inner tolerance of dd_eigenpair).
int batched_ipm(dd_batch* b, double* lambda_out, int* outer_out, int* inner_out, double* seconds_out,
                const std::vector<double>& setup_s, std::chrono::steady_clock::time_point t_start) {
  const int n = (int)b->ctx.size();
  const double tol_res = 1e-8, tol_lam = 1e-10, rtol_inner = 1e-8;
  const int maxit_outer = 100, maxit_inner = 10000;
  if (!b->built) build_engine(b);
  if (!b->graph) build_graph(b);
  std::vector<double> rho_prev(n), rho(n, 0.0);
  std::vector<int> outer(n, 0), inner_tot(n, 0), status(n, DD_OK);
  for (int i = 0; i < n; ++i) {
    b->Bh[i].active = 1;
    DD_CUDA(cudaMemsetAsync(b->ctx[i]->ost, 0, sizeof(dd::OuterState), b->s));
  }
  upload_active(b);
  // x_0 -> M-normalised iterate, its images
  dd::launch_b_pad(b->B, b->vm_vec, b->n_vec, b->xptr_d, dd::BV_W1, b->s);
  outer_images(b, dd::BV_W1);
  gather(b);
  int active = 0;
  for (int i = 0; i < n; ++i) {
    if (b->stat_h[i].outer_status != 0) {
      status[i] = b->stat_h[i].outer_status;
      b->Bh[i].active = 0;
      continue;
    }
    rho_prev[i] = b->ctx[i]->sigma + b->stat_h[i].xAx;
    rho[i] = rho_prev[i];
    ++active;
  }
  upload_active(b);
  for (int k = 1; k <= maxit_outer && active > 0; ++k) {
    // A_sigma w = M x_k by PCG from zero, every active instance
    dd::launch_b_zero_pcg(b->B, b->vm_vec, b->n_vec, b->s);
    dd::launch_b_pcg_reset(b->B, n, rtol_inner * rtol_inner, maxit_inner, b->s);
    dd::launch_b_pcg_init(b->B, b->vm_init, b->n_init, dd::BV_W2, b->s);
    precond(b, 1);
    for (int done_iters = 0; done_iters < maxit_inner + b->check_every; done_iters += b->check_every) {
      DD_CUDA(cudaGraphLaunch(b->graph, b->s));
      dd::note_launches(b->graph_kernels);
      gather(b);
      bool all = true;
      for (int i = 0; i < n; ++i)
        if (b->Bh[i].active && !b->stat_h[i].pcg_done) all = false;
      if (all) break;
    }
    for (int i = 0; i < n; ++i) {
      if (!b->Bh[i].active) continue;
      inner_tot[i] += b->stat_h[i].pcg_iter;
      const int ps = b->stat_h[i].pcg_status;
      if (ps != 0 && ps != DD_EMAXIT) {
        status[i] = ps;
        b->Bh[i].active = 0;
        outer[i] = k;
      }
    }
    upload_active(b);
    outer_images(b, dd::BV_X);
    gather(b);
    const double now = std::chrono::duration<double>(std::chrono::steady_clock::now() - t_start).count();
    active = 0;
    for (int i = 0; i < n; ++i) {
      if (!b->Bh[i].active) continue;
      const BStat& h = b->stat_h[i];
      outer[i] = k;
      if (h.outer_status != 0) {
        status[i] = h.outer_status;
        b->Bh[i].active = 0;
        continue;
      }
      rho[i] = b->ctx[i]->sigma + h.xAx;
      const double eta = std::sqrt(h.rr / h.mm) / std::fabs(rho[i]);
      if (!std::isfinite(rho[i])) {
        status[i] = DD_ENAN;
        b->Bh[i].active = 0;
      } else if (eta <= tol_res && std::fabs(rho[i] - rho_prev[i]) <= tol_lam * std::fabs(rho[i])) {
        b->Bh[i].active = 0;
        if (seconds_out) seconds_out[i] = setup_s[i] + now;
      } else {
        rho_prev[i] = rho[i];
        ++active;
        if (k == maxit_outer) status[i] = DD_EMAXIT;
      }
    }
    upload_active(b);
  }
  // phi (M-normalised iterate) back to the instances' vectors
  dd::launch_b_unpad(b->B, b->vm_vec, b->n_vec, dd::BV_XE, b->xptr_d, b->s);
  int herr = 0;
  DD_CUDA(cudaMemcpyAsync(&herr, b->err_d + 8, sizeof(int), cudaMemcpyDeviceToHost, b->s));
  DD_CUDA(cudaStreamSynchronize(b->s));
  const double end = std::chrono::duration<double>(std::chrono::steady_clock::now() - t_start).count();
  int first = DD_OK;
  for (int i = 0; i < n; ++i) {
    if (lambda_out) lambda_out[i] = rho[i];
    if (outer_out) outer_out[i] = outer[i];
    if (inner_out) inner_out[i] = inner_tot[i];
    if (seconds_out && status[i] != DD_OK) seconds_out[i] = setup_s[i] + end;
    if (status[i] != DD_OK && first == DD_OK) first = status[i];
  }
  if (herr != 0) {
    DD_CUDA(cudaMemsetAsync(b->err_d + 8, 0, sizeof(int), b->s));
    return DD_ETIMEOUT;
  }
  return first;
}

// the SI-LOPCG work space of every instance (what dd_lopcg allocates on its first call)
void ensure_lopcg(dd_batch* b) {
  for (size_t i = 0; i < b->ctx.size(); ++i) {
    dd_ctx* c = b->ctx[i];
    if (!c->lst) {
      c->lst = (dd::LopState*)dd::dev_alloc(c, sizeof(dd::LopState));
      DD_CUDA(cudaMallocHost(&c->lst_h, sizeof(dd::LopState)));
      c->lop_red = (double*)dd::dev_alloc(c, sizeof(double) * dd::kMaxRedBlocksHost * 15);
      for (double*& v : c->lop) v = dd::alloc_vec(c);
      DD_CUDA(cudaStreamSynchronize(c->stream));
    }
    BInst& I = b->Bh[i];
    for (int k = 0; k < 12; ++k) I.lop[k] = c->lop[k];
    I.lst = c->lst;
    I.lop_red = c->lop_red;
  }
}

// Batched SI-LOPCG with the fused inner step (Algorithm 1 with w_k = M_AS2^{-1} r_o, Sec. 4.3),
// the steps of dd_lopcg for every active instance at once.  The twelve work vectors play the
// same roles in every instance (the roles rotate in lockstep), so each launch names roles.
int batched_lopcg_fused(dd_batch* b, double* lambda_out, int* outer_out, int* inner_out, double* seconds_out,
                        const std::vector<double>& setup_s, std::chrono::steady_clock::time_point t_start) {
  using namespace dd;
  const int n = (int)b->ctx.size();
  const double tol_res = 1e-8, tol_lam = 1e-10;
  const int maxit_outer = 1000;
  if (!b->built) build_engine(b);
  ensure_lopcg(b);
  for (int i = 0; i < n; ++i) {
    b->Bh[i].active = 1;
    b->Bh[i].r = b->ctx[i]->lop[9];   // the preconditioner is applied to the outer residual r_o
  }
  upload_active(b);
  // roles: X XP T AX AXP MX MXP AW MW RO AT MT = lop[0..11] at the start
  int X = 0, XP = 1, T = 2, AX = 3, AXP = 4, MX = 5, MXP = 6;
  const int AW = 7, MW = 8, RO = 9;
  int AT = 10, MT = 11;
  auto R = [](int k) { return BV_LOP + k; };
  cudaStream_t s = b->s;
  launch_b_zero_roles(b->B, b->vm_vec, b->n_vec, BV_LOP, 12, s);
  launch_b_lop_reset(b->B, n, s);
  const long long first = (long long)b->ctx.front()->g.Ypad;   // first interior node (p = 1)
  launch_b_set_entry(b->B, n, R(XP), first, 1.0, s);
  launch_b_stencil_role(b->B, b->vm_st, b->n_st, 1, R(XP), R(MXP), s);
  launch_b_lop_normalize(b->B, b->vm_vec, b->n_vec, R(XP), R(MXP), s);
  launch_b_stencil_role(b->B, b->vm_st, b->n_st, 0, R(XP), R(AXP), s);
  auto explicit_images = [&]() {
    launch_b_stencil_role(b->B, b->vm_st, b->n_st, 1, R(X), R(MX), s);
    launch_b_lop_normalize(b->B, b->vm_vec, b->n_vec, R(X), R(MX), s);
    launch_b_stencil_dot(b->B, b->vm_sdot, b->n_sdot, R(X), R(AX), s);
    launch_b_outer_res_ro(b->B, b->vm_vec, b->n_vec, R(AX), R(MX), R(RO), s);
    gather(b);
  };
  launch_b_pad(b->B, b->vm_vec, b->n_vec, b->xptr_d, R(X), s);
  explicit_images();
  std::vector<double> lam(n), rr(n), mm(n), rho(n), rho_prev(n, std::numeric_limits<double>::infinity());
  std::vector<int> exact(n, 1), outer(n, 0), inner(n, 0), status(n, DD_OK), xrole(n, X);
  for (int i = 0; i < n; ++i) {
    if (b->stat_h[i].outer_status != 0) {
      status[i] = b->stat_h[i].outer_status;
      b->Bh[i].active = 0;
      continue;
    }
    lam[i] = b->stat_h[i].xAx;
    rr[i] = b->stat_h[i].rr;
    mm[i] = b->stat_h[i].mm;
  }
  upload_active(b);
  auto stops = [&](double rh, double r2, double m2, double prev) {
    const double eta = std::sqrt(r2 / m2) / std::fabs(rh);
    return eta <= tol_res && std::fabs(rh - prev) <= tol_lam * std::fabs(rh);
  };
  for (int k = 0; k <= maxit_outer; ++k) {
    // stop test; instances whose images are carried combinations confirm on recomputed ones
    std::vector<int> confirm;
    int active = 0;
    for (int i = 0; i < n; ++i) {
      if (!b->Bh[i].active) continue;
      rho[i] = b->ctx[i]->sigma + lam[i];
      if (!std::isfinite(rho[i])) {
        status[i] = DD_ENAN;
        b->Bh[i].active = 0;
        continue;
      }
      if (stops(rho[i], rr[i], mm[i], rho_prev[i])) {
        if (exact[i]) {
          b->Bh[i].active = 0;
          outer[i] = k;
          xrole[i] = X;
          if (seconds_out)
            seconds_out[i] = setup_s[i] + std::chrono::duration<double>(std::chrono::steady_clock::now() - t_start).count();
          continue;
        }
        confirm.push_back(i);
      }
      ++active;
    }
    if (!confirm.empty()) {
      std::vector<int> keep(n);
      for (int i = 0; i < n; ++i) {
        keep[i] = b->Bh[i].active;
        b->Bh[i].active = 0;
      }
      for (int i : confirm) b->Bh[i].active = 1;
      upload_active(b);
      explicit_images();
      for (int i = 0; i < n; ++i) b->Bh[i].active = keep[i];
      for (int i : confirm) {
        exact[i] = 1;
        lam[i] = b->stat_h[i].xAx;
        rr[i] = b->stat_h[i].rr;
        mm[i] = b->stat_h[i].mm;
        const double rho_e = b->ctx[i]->sigma + lam[i];
        if (stops(rho_e, rr[i], mm[i], rho_prev[i])) {
          rho[i] = rho_e;
          b->Bh[i].active = 0;
          outer[i] = k;
          xrole[i] = X;
          --active;
          if (seconds_out)
            seconds_out[i] = setup_s[i] + std::chrono::duration<double>(std::chrono::steady_clock::now() - t_start).count();
        }
      }
      upload_active(b);
    }
    if (active == 0) break;
    if (k == maxit_outer) {
      for (int i = 0; i < n; ++i)
        if (b->Bh[i].active) {
          status[i] = DD_EMAXIT;
          outer[i] = k;
          xrole[i] = X;
        }
      break;
    }
    // w = M_AS2^{-1} r_o; images of w; Rayleigh-Ritz on span{x_k, w, x_{k-1}}; update
    launch_b_pcg_reset(b->B, n, 0.0, 0, s);
    precond(b, 0);
    launch_b_stencil2(b->B, b->vm_st2, b->n_st2, BV_Z, R(AW), R(MW), s);
    const int S[3] = {R(X), BV_Z, R(XP)}, AS[3] = {R(AX), R(AW), R(AXP)}, MS[3] = {R(MX), R(MW), R(MXP)};
    launch_b_lop_gram(b->B, b->vm_vec, b->n_vec, S, AS, MS, 1e-10, s);
    launch_b_lop_update3(b->B, b->vm_vec, b->n_vec, S, AS, MS, R(T), R(AT), R(MT), R(RO), s);
    int t0 = XP;
    XP = X; X = T; T = t0;
    t0 = AXP; AXP = AX; AX = AT; AT = t0;
    t0 = MXP; MXP = MX; MX = MT; MT = t0;
    gather(b);
    for (int i = 0; i < n; ++i) {
      if (!b->Bh[i].active) continue;
      inner[i] += 1;
      if (b->stat_h[i].lop_status != 0) {
        status[i] = b->stat_h[i].lop_status;
        b->Bh[i].active = 0;
        outer[i] = k + 1;
        xrole[i] = X;
        continue;
      }
      rho_prev[i] = rho[i];
      lam[i] = b->stat_h[i].theta;
      rr[i] = b->stat_h[i].lop_rr;
      mm[i] = b->stat_h[i].lop_mm;
      exact[i] = 0;
    }
    upload_active(b);
  }
  // phi back to the instances' vectors: each from the role its iterate had when it stopped
  for (int role = 0; role < 12; ++role) {
    bool any = false;
    for (int i = 0; i < n; ++i) {
      b->Bh[i].active = (xrole[i] == role) ? 1 : 0;
      any = any || xrole[i] == role;
    }
    if (!any) continue;
    upload_active(b);
    launch_b_unpad_active(b->B, b->vm_vec, b->n_vec, R(role), b->xptr_d, s);
  }
  for (int i = 0; i < n; ++i) b->Bh[i].r = b->ctx[i]->r;
  upload_active(b);
  int herr = 0;
  DD_CUDA(cudaMemcpyAsync(&herr, b->err_d + 8, sizeof(int), cudaMemcpyDeviceToHost, s));
  DD_CUDA(cudaStreamSynchronize(s));
  const double end = std::chrono::duration<double>(std::chrono::steady_clock::now() - t_start).count();
  int first_err = DD_OK;
  for (int i = 0; i < n; ++i) {
    if (lambda_out) lambda_out[i] = rho[i];
    if (outer_out) outer_out[i] = std::min(outer[i], maxit_outer);
    if (inner_out) inner_out[i] = inner[i];
    if (seconds_out && status[i] != DD_OK) seconds_out[i] = setup_s[i] + end;
    if (status[i] != DD_OK && first_err == DD_OK) first_err = status[i];
  }
  if (herr != 0) {
    DD_CUDA(cudaMemsetAsync(b->err_d + 8, 0, sizeof(int), s));
    return DD_ETIMEOUT;
  }
  return first_err;
}

}  // namespace

extern "C" {

int dd_batch_create(const dd_grid* grids, const double* const* V, const size_t* nV, int count, void* stream,
                    dd_batch** out) {
  if (out) *out = nullptr;
  if (!grids || !V || !nV || !out || count < 1) return DD_EINVAL;
  dd_batch* b = new (std::nothrow) dd_batch();
  if (!b) return DD_ENOMEM;
  cudaGetDevice(&b->device);
  for (int i = 0; i < count; ++i) {
    dd_ctx* c = nullptr;
    const int rc = dd_setup(&grids[i], V[i], nV[i], stream, &c);
    if (rc != DD_OK) {
      destroy_all(b);
      return rc;
    }
    b->ctx.push_back(c);
    dd_info info;
    dd_query(c, &info);
    b->ndof.push_back(info.ndof);
    double* x = nullptr;
    if (cudaMalloc(&x, sizeof(double) * (size_t)info.ndof) != cudaSuccess) {
      cudaGetLastError();
      destroy_all(b);
      return DD_ENOMEM;
    }
    b->x.push_back(x);
  }
  // batch-wide buffers of the grouped contraction; each context computes into its rows
  b->eligible = batchable(b);
  if (b->eligible) {
    b->precision = b->ctx.front()->grid.precision;
    const size_t es = b->precision == DD_PREC_BF16 ? 2 : 4;
    const size_t kpad = (size_t)b->ctx.front()->kpad;
    int types = 0, slots = 0;
    for (dd_ctx* c : b->ctx) {
      b->type_base.push_back(types);
      b->slot_base.push_back(slots);
      types += c->ntypes;
      slots += c->g.nsub;
    }
    const size_t ba = es * types * kpad * kpad, br = es * slots * kpad, by = sizeof(float) * slots * kpad;
    if (cudaMalloc(&b->Ainv_all, ba) != cudaSuccess || cudaMalloc(&b->Rpack_all, br) != cudaSuccess ||
        cudaMalloc((void**)&b->Y_all, by) != cudaSuccess) {
      cudaGetLastError();
      destroy_all(b);
      return DD_ENOMEM;
    }
    cudaMemset(b->Ainv_all, 0, ba);
    cudaMemset(b->Rpack_all, 0, br);
    cudaMemset(b->Y_all, 0, by);
    for (size_t i = 0; i < b->ctx.size(); ++i) {
      dd_ctx* c = b->ctx[i];
      c->Ainv = (char*)b->Ainv_all + es * (size_t)b->type_base[i] * kpad * kpad;
      c->Rpack = (char*)b->Rpack_all + es * (size_t)b->slot_base[i] * kpad;
      c->Y32 = b->Y_all + (size_t)b->slot_base[i] * kpad;
    }
  }
  *out = b;
  return DD_OK;
}

int dd_batch_size(const dd_batch* b) { return b ? (int)b->ctx.size() : 0; }

int dd_batch_info(const dd_batch* b, int* batchable_out, int* last_batched_out, int* gemm_tile_n_out,
                  int* check_every_out) {
  if (!b) return DD_EINVAL;
  if (batchable_out) *batchable_out = b->eligible ? 1 : 0;
  if (last_batched_out) *last_batched_out = b->last_batched;
  if (gemm_tile_n_out) *gemm_tile_n_out = b->bn;
  if (check_every_out) *check_every_out = b->check_every;
  return DD_OK;
}

dd_ctx* dd_batch_context(dd_batch* b, int i) {
  if (!b || i < 0 || i >= (int)b->ctx.size()) return nullptr;
  return b->ctx[i];
}

int dd_batch_ground_states(dd_batch* b, int method, int threads, double* lambda_out, double* const* phi_out,
                           int* outer_out, int* inner_out, double* seconds_out) {
  if (!b) return DD_EINVAL;
  if (method < DD_BATCH_IPM || method > DD_BATCH_IPM_CONCURRENT) return DD_EINVAL;
  const int n = (int)b->ctx.size();
  b->last_batched = 0;
  if (threads < 1) threads = std::min(n, 16);
  threads = std::min(threads, n);
  // the batched engine needs the options it was built for (the grouped contraction and
  // the cyclic-reduction coarse solve, PCG inner solves)
  bool engine = b->eligible && (method == DD_BATCH_IPM || method == DD_BATCH_LOPCG_FUSED);
  for (dd_ctx* c : b->ctx)
    if (c->krylov != 0 || c->ras != 0 || c->coarse_mode == 2 || c->timing) engine = false;
  std::vector<int> order(n);
  for (int i = 0; i < n; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](int a, int c) { return b->ndof[a] > b->ndof[c]; });
  std::atomic<int> next{0};
  std::atomic<int> first_error{DD_OK};
  std::vector<double> setup_s(n, 0.0);
  const auto t_start = std::chrono::steady_clock::now();
  auto worker = [&]() {
    cudaSetDevice(b->device);
    cudaStream_t s = nullptr;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) {
      cudaGetLastError();
      int expect = DD_OK;
      first_error.compare_exchange_strong(expect, DD_ECUDA);
      return;
    }
    for (int k = next.fetch_add(1); k < n; k = next.fetch_add(1)) {
      const int i = order[k];
      dd_ctx* c = b->ctx[i];
      double lam = 0.0;
      int outer = 0, tot = 0, mx = 0;
      int rc = dd_cell_eigenpair(c, nullptr, nullptr);
      if (rc == DD_OK) rc = dd_coarse_build(c);
      if (rc == DD_OK) {
        (k_fill<<<64, 256, 0, s>>>(b->ndof[i], 1.0, b->x[i]), dd::note_launch());
        if (cudaStreamSynchronize(s) != cudaSuccess) {
          cudaGetLastError();
          rc = DD_ECUDA;
        }
      }
      setup_s[i] = std::chrono::duration<double>(std::chrono::steady_clock::now() - t_start).count();
      if (rc == DD_OK && !engine) {
        if (method == DD_BATCH_IPM || method == DD_BATCH_IPM_CONCURRENT)
          rc = dd_inverse_iterate(c, b->x[i], 1e-8, 1e-10, 100, 1e-8, &lam, &outer, &tot, &mx);
        else
          rc = dd_lopcg(c, b->x[i], method == DD_BATCH_LOPCG_FUSED ? DD_INNER_FUSED : DD_INNER_ADAPTIVE, 1e-8,
                        1e-10, 1000, 1e-8, &lam, &outer, &tot, &mx);
        if (lambda_out) lambda_out[i] = lam;
        if (outer_out) outer_out[i] = outer;
        if (inner_out) inner_out[i] = tot;
        if (seconds_out)
          seconds_out[i] = std::chrono::duration<double>(std::chrono::steady_clock::now() - t_start).count();
      }
      if (rc != DD_OK) {
        int expect = DD_OK;
        first_error.compare_exchange_strong(expect, rc);
      }
    }
    cudaStreamDestroy(s);
  };
  std::vector<std::thread> pool;
  pool.reserve(threads);
  for (int t = 0; t < threads; ++t) pool.emplace_back(worker);
  for (auto& th : pool) th.join();
  int rc = first_error.load();
  if (rc == DD_OK && engine) {
    // every instance's set-up is complete (each call synchronised its context's stream)
    try {
      DD_CUDA(cudaSetDevice(b->device));
      rc = method == DD_BATCH_IPM
               ? batched_ipm(b, lambda_out, outer_out, inner_out, seconds_out, setup_s, t_start)
               : batched_lopcg_fused(b, lambda_out, outer_out, inner_out, seconds_out, setup_s, t_start);
      b->last_batched = 1;
      // bounded waits of the instances' coarse solves
      for (dd_ctx* c : b->ctx) {
        int e = 0;
        DD_CUDA(cudaMemcpy(&e, c->dev_err + 8, sizeof(int), cudaMemcpyDeviceToHost));
        if (e != 0) {
          DD_CUDA(cudaMemset(c->dev_err + 8, 0, sizeof(int)));
          if (rc == DD_OK) rc = DD_ETIMEOUT;
        }
      }
    } catch (const dd::Error& e) {
      b->err = e.msg;
      rc = e.code;
    } catch (...) {
      rc = DD_ECUDA;
    }
  }
  if (phi_out) {
    for (int i = 0; i < n; ++i) {
      if (!phi_out[i]) continue;
      if (cudaMemcpy(phi_out[i], b->x[i], sizeof(double) * (size_t)b->ndof[i], cudaMemcpyDefault) != cudaSuccess) {
        cudaGetLastError();
        if (rc == DD_OK) rc = DD_ECUDA;
      }
    }
  }
  return rc;
}

void dd_batch_destroy(dd_batch* b) {
  if (b) destroy_all(b);
}

}  // extern "C"
