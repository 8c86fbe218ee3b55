// Batched ground states: many independent instances (uneven L, own potential and shift).
//
// Set-up (cell eigenpair, local inverses, coarse matrix) runs per instance, each on its own
// context and private stream, on a pool of host threads (largest instance first); its cost
// does not grow with L.
//
// The eigen-iteration runs batched when the instances share everything but L, the potential
// and the shift (p = 1, rounded local inverses, same h, delta, ell, quadrature and partition
// of unity).  The instances are split into G groups of about equal total size; each group is
// driven by one host thread on its own streams, and within a group every kernel of an
// iteration is ONE launch over all of the group's instances -- its blocks are the blocks of
// each instance's own launch (block index and count within the instance), the local solves
// one grouped tensor-core contraction over the instances' tiles -- and a block of PCG
// iterations is one CUDA graph.  Each instance keeps its own device scalars (PCG state, outer
// state); kernels of an instance whose solve is done return at once; an instance joins its
// group's iteration as soon as its own set-up is done and drops out when its eigen-iteration
// stops, so set-up and solves overlap.  Groups run side by side, so the GPU interleaves their
// kernel types (FP64 stencils, HBM-bound updates, tensor-core contractions) as concurrent
// pipelines do.  G is chosen by timing (every G gives the same bits).  Results equal those of
// the single-instance calls bit for bit.  Other combinations (p = 2, the plain FP64 form,
// adaptive SI-LOPCG) run as concurrent per-instance pipelines.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstring>
#include <limits>
#include <map>
#include <mutex>
#include <thread>
#include <vector>

#include "dd_internal.h"

namespace {

using dd::BInst;
using dd::BStat;

enum { ST_PENDING = 0, ST_RUNNING = 1, ST_DONE = 2 };

// One group of instances run as batched launches (its own streams, graph, contraction).
struct BGroup {
  std::vector<int> idx;            // the batch's instance indices in this group (ascending)
  std::vector<BInst> Bh;
  BInst* B = nullptr;
  int2 *vm_init = nullptr, *vm_fused = nullptr, *vm_xr = nullptr, *vm_prolong = nullptr, *vm_sdot = nullptr,
       *vm_st = nullptr, *vm_st2 = nullptr, *vm_vec = nullptr, *vm_pack = nullptr;
  int n_init = 0, n_fused = 0, n_xr = 0, n_prolong = 0, n_sdot = 0, n_st = 0, n_st2 = 0, n_vec = 0, n_pack = 0;
  size_t cr_smem = 0;
  int ypad = 0, precision = 0, check_every = 8;
  bool arith = true;               // every instance's prolong-sum owners in closed form
  bool pairs = false;              // q = A_sigma p in float pairs (the same choice for every instance)
  bool fuse = false;               // the x/r update inside the packing (the same for every instance)
  dd::BGemm* gemm = nullptr;
  int bn = 0;                      // N tile of the grouped contraction (timed at build)
  cudaStream_t s = nullptr, side = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  cudaGraphExec_t graph = nullptr;
  long long graph_kernels = 0;
  BStat* stat_d = nullptr;
  BStat* stat_h = nullptr;
  double** xptr_d = nullptr;       // the instances' start / solution vectors
  int* err_d = nullptr;            // error word of the grouped contraction's bounded waits
};

}  // namespace

struct dd_batch {
  std::vector<dd_ctx*> ctx;
  std::vector<double*> x;      // per instance: device start vector / solution (ndof)
  std::vector<long long> ndof;
  int device = 0;

  bool eligible = false;
  int precision = 0;
  void* Ainv_all = nullptr;    // [sum of types][kpad][kpad] rounded local inverses
  void* Rpack_all = nullptr;   // [sum of subdomains][kpad] packed restrictions
  float* Y_all = nullptr;      // [sum of subdomains][kpad] local solutions
  std::vector<int> type_base, slot_base;
  std::map<int, std::vector<BGroup*>> engines;   // built groups, per group count
  std::map<long long, double> timed;              // (method, groups) -> best call seconds
  int groups_opt = 0;          // 0: chosen by timing; > 0: fixed
  long long opt_sig = -1;      // the instances' options the built groups were made for
  int last_batched = 0, last_groups = 0, last_bn = 0;
  double last_setup_s = 0.0, last_total_s = 0.0;
};

namespace {

__global__ void k_fill(long long n, double v, double* x) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n;
       t += (long long)gridDim.x * blockDim.x)
    x[t] = v;
}

void free_group(BGroup* g) {
  if (!g) return;
  if (g->graph) cudaGraphExecDestroy(g->graph);
  dd::bgemm_destroy(g->gemm);
  for (void* p : {(void*)g->B, (void*)g->vm_init, (void*)g->vm_fused, (void*)g->vm_xr, (void*)g->vm_prolong,
                  (void*)g->vm_sdot, (void*)g->vm_st, (void*)g->vm_st2, (void*)g->vm_vec, (void*)g->vm_pack,
                  (void*)g->stat_d, (void*)g->xptr_d, (void*)g->err_d})
    if (p) cudaFree(p);
  if (g->stat_h) cudaFreeHost(g->stat_h);
  if (g->side) cudaStreamDestroy(g->side);
  if (g->s) cudaStreamDestroy(g->s);
  if (g->ev_fork) cudaEventDestroy(g->ev_fork);
  if (g->ev_join) cudaEventDestroy(g->ev_join);
  delete g;
}

// The per-instance options a built group bakes in; a change on any instance's context
// (dd_batch_context + dd_set_option) drops the built groups and their timings.
long long option_signature(const dd_batch* b) {
  long long h = 1469598103934665603LL;
  for (const dd_ctx* c : b->ctx)
    for (int v : {c->prolong_arith, c->pq_pairs, c->fuse_xr, c->flexible_opt, c->check_every, c->gemm_bn_opt})
      h = (h ^ (long long)(v + 7)) * 1099511628211LL;
  return h;
}

void drop_engines(dd_batch* b) {
  for (auto& kv : b->engines)
    for (BGroup* g : kv.second) free_group(g);
  b->engines.clear();
  b->timed.clear();
}

void destroy_all(dd_batch* b) {
  for (auto& kv : b->engines)
    for (BGroup* g : kv.second) free_group(g);
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

void upload(BGroup* g) {
  DD_CUDA(cudaMemcpyAsync(g->B, g->Bh.data(), sizeof(BInst) * g->Bh.size(), cudaMemcpyHostToDevice, g->s));
}

template <typename F>
void mask(BGroup* g, F&& on) {
  for (size_t j = 0; j < g->Bh.size(); ++j) g->Bh[j].active = on((int)j) ? 1 : 0;
  upload(g);
}

// z = M_AS2^{-1} r for every active instance (mode 0: alone, 1: PCG start, 2: iteration); the
// coarse solves run on the side stream beside the grouped contraction (the operator is additive)
// (packed: the restrictions came from the fused x/r update, whose r update the prolong-sum applies)
void precond(BGroup* g, int mode, bool packed = false) {
  if (!packed) dd::launch_b_pack(g->B, g->vm_pack, g->n_pack, g->precision, g->s);
  DD_CUDA(cudaEventRecord(g->ev_fork, g->s));
  DD_CUDA(cudaStreamWaitEvent(g->side, g->ev_fork, 0));
  dd::launch_b_cr_solve(g->B, (int)g->idx.size(), g->cr_smem, g->side);
  DD_CUDA(cudaEventRecord(g->ev_join, g->side));
  dd::bgemm_run(g->gemm, g->bn, g->s);
  DD_CUDA(cudaStreamWaitEvent(g->s, g->ev_join, 0));
  dd::launch_b_prolong(g->B, g->vm_prolong, g->n_prolong, mode, g->arith, packed, g->s);
}

void pcg_iteration(BGroup* g) {
  dd::launch_b_fused_pq(g->B, g->vm_fused, g->n_fused, g->ypad, g->pairs, g->s);
  if (g->fuse) {
    dd::launch_b_pack_xr(g->B, g->vm_pack, g->n_pack, g->precision, g->s);
    precond(g, 2, true);
  } else {
    dd::launch_b_xr_update(g->B, g->vm_xr, g->n_xr, g->s);
    precond(g, 2);
  }
}

void build_graph(BGroup* g) {
  cudaGraph_t gr;
  DD_CUDA(cudaStreamBeginCapture(g->s, cudaStreamCaptureModeThreadLocal));
  dd::set_capturing(true);
  try {
    for (int i = 0; i < g->check_every; ++i) pcg_iteration(g);
  } catch (...) {
    dd::set_capturing(false);
    cudaStreamEndCapture(g->s, &gr);
    cudaGetLastError();
    throw;
  }
  dd::set_capturing(false);
  DD_CUDA(cudaStreamEndCapture(g->s, &gr));
  g->graph_kernels = dd::graph_kernel_nodes(gr);   // replays are counted when launched
  DD_CUDA(cudaGraphInstantiate(&g->graph, gr, 0));
  DD_CUDA(cudaGraphDestroy(gr));
}

// the SI-LOPCG work space of every instance (what dd_lopcg allocates on its first call); the
// calling thread must be the only one using the contexts
void ensure_lopcg(dd_batch* b) {
  for (dd_ctx* c : b->ctx) {
    if (c->lst) continue;
    c->lst = (dd::LopState*)dd::dev_alloc(c, sizeof(dd::LopState));
    DD_CUDA(cudaMallocHost(&c->lst_h, sizeof(dd::LopState)));
    c->lop_red = (double*)dd::dev_alloc(c, sizeof(double) * dd::kMaxRedBlocksHost * 15);
    for (double*& v : c->lop) v = dd::alloc_vec(c);
    DD_CUDA(cudaStreamSynchronize(c->stream));
  }
}

// Descriptors, block maps, streams, graph and grouped contraction of one group (every
// instance of the group set up; its N tile timed on the group's own operands).
BGroup* build_group(dd_batch* b, const std::vector<int>& idx) {
  BGroup* g = new BGroup();
  try {
    g->idx = idx;
    g->precision = b->precision;
    const int n = (int)idx.size();
    DD_CUDA(cudaSetDevice(b->device));
    DD_CUDA(cudaStreamCreateWithFlags(&g->s, cudaStreamNonBlocking));
    DD_CUDA(cudaStreamCreateWithFlags(&g->side, cudaStreamNonBlocking));
    DD_CUDA(cudaEventCreateWithFlags(&g->ev_fork, cudaEventDisableTiming));
    DD_CUDA(cudaEventCreateWithFlags(&g->ev_join, cudaEventDisableTiming));
    DD_CUDA(cudaMalloc(&g->err_d, sizeof(int) * 16));
    DD_CUDA(cudaMemset(g->err_d, 0, sizeof(int) * 16));
    g->Bh.assign(n, BInst());
    std::vector<int2> vinit, vfused, vxr, vprol, vsdot, vst, vst2, vvec, vpack;
    std::vector<dd_ctx*> cs;
    std::vector<int> tb, sb;
    std::vector<double*> xs;
    for (int j = 0; j < n; ++j) {
      const int i = idx[j];
      dd_ctx* c = b->ctx[i];
      cs.push_back(c);
      tb.push_back(b->type_base[i]);
      sb.push_back(b->slot_base[i]);
      xs.push_back(b->x[i]);
      BInst& I = g->Bh[j];
      std::memset(&I, 0, sizeof(I));
      I.g = c->g;
      I.x = c->x; I.r = c->r; I.z = c->z; I.pb0 = c->pb[0]; I.pb1 = c->pb[1]; I.q = c->q;
      I.w1 = c->w1; I.w2 = c->w2; I.w3 = c->w3; I.xe = c->xe;
      I.tabS = c->tabS; I.tabM = c->tabM;
      I.tabS2 = c->tabS2;
      I.pq_pairs = c->pq_pairs;
      g->pairs = c->pq_pairs != 0;
      g->fuse = c->fuse_xr != 0;
      I.st = c->st; I.ost = c->ost; I.red = c->red; I.cnt = c->cnt;
      I.subs = c->subs; I.slot_of_sub = c->slot_of_sub; I.Rpack = c->Rpack; I.wT = c->wT; I.c0 = c->c0;
      I.u0 = c->u0; I.u0f = c->u0f; I.Y32 = c->Y32; I.wT32 = c->wT32; I.puT32 = c->puT32;
      I.axown = c->axown; I.subrow = c->subrow; I.colrow = c->colrow; I.cr = c->cr;
      I.cr_m = c->cr_m; I.cr_c2 = c->cr_c2; I.cr_w2 = c->cr_w2;
      size_t smem = 0;
      int staged = 0;
      dd::cr_launch_shape(c, &smem, &staged);
      I.cr_staged = staged;
      g->cr_smem = std::max(g->cr_smem, smem);
      I.kpad = c->kpad; I.coarse = 1; I.nsub = c->g.nsub;
      I.flexible = (c->flexible_opt < 0) ? 1 : c->flexible_opt;
      I.err = c->dev_err;
      I.active = 1;
      I.ptypes = c->ptypes;
      I.prolong_arith = c->prolong_arith;
      g->arith = g->arith && c->prolong_arith;
      dd::batch_grid_sizes(c, &I);
      for (int k = 0; k < I.nb_init; ++k) vinit.push_back(make_int2(j, k));
      for (int k = 0; k < I.nb_fused; ++k) vfused.push_back(make_int2(j, k));
      for (int k = 0; k < I.nb_xr; ++k) vxr.push_back(make_int2(j, k));
      for (int k = 0; k < I.nb_prolong; ++k) vprol.push_back(make_int2(j, k));
      for (int k = 0; k < I.nb_sdot; ++k) vsdot.push_back(make_int2(j, k));
      for (int k = 0; k < I.nb_st; ++k) vst.push_back(make_int2(j, k));
      for (int k = 0; k < I.nb_st2; ++k) vst2.push_back(make_int2(j, k));
      for (int k = 0; k < I.nb_vec; ++k) vvec.push_back(make_int2(j, k));
      for (int k = 0; k < c->g.nsub; ++k) vpack.push_back(make_int2(j, k));
    }
    if (g->cr_smem > 220 * 1024) throw dd::Error(DD_EINVAL, "coarse chain too long for the batched cyclic reduction");
    g->ypad = b->ctx.front()->g.Ypad;
    g->vm_init = upload_vmap(vinit); g->n_init = (int)vinit.size();
    g->vm_fused = upload_vmap(vfused); g->n_fused = (int)vfused.size();
    g->vm_xr = upload_vmap(vxr); g->n_xr = (int)vxr.size();
    g->vm_prolong = upload_vmap(vprol); g->n_prolong = (int)vprol.size();
    g->vm_sdot = upload_vmap(vsdot); g->n_sdot = (int)vsdot.size();
    g->vm_st = upload_vmap(vst); g->n_st = (int)vst.size();
    g->vm_st2 = upload_vmap(vst2); g->n_st2 = (int)vst2.size();
    g->vm_vec = upload_vmap(vvec); g->n_vec = (int)vvec.size();
    g->vm_pack = upload_vmap(vpack); g->n_pack = (int)vpack.size();
    DD_CUDA(cudaMalloc(&g->B, sizeof(BInst) * n));
    DD_CUDA(cudaMemcpy(g->B, g->Bh.data(), sizeof(BInst) * n, cudaMemcpyHostToDevice));
    DD_CUDA(cudaMalloc(&g->stat_d, sizeof(BStat) * n));
    DD_CUDA(cudaMallocHost(&g->stat_h, sizeof(BStat) * n));
    DD_CUDA(cudaMalloc(&g->xptr_d, sizeof(double*) * n));
    DD_CUDA(cudaMemcpy(g->xptr_d, xs.data(), sizeof(double*) * n, cudaMemcpyHostToDevice));
    g->gemm = dd::bgemm_create(cs, tb, sb, b->Ainv_all, b->Rpack_all, b->Y_all, g->err_d + 8, g->s);
    dd::launch_b_pcg_reset(g->B, n, 1.0, 1, g->s);   // done flags cleared for the timing
    g->bn = dd::bgemm_tune(g->gemm, g->s);
    build_graph(g);
    DD_CUDA(cudaStreamSynchronize(g->s));
  } catch (...) {
    free_group(g);
    throw;
  }
  return g;
}

// G groups of about equal total size: instances largest first, each to the lightest group
std::vector<std::vector<int>> partition(const dd_batch* b, int G) {
  const int n = (int)b->ctx.size();
  std::vector<int> order(n);
  for (int i = 0; i < n; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](int a, int c) { return b->ndof[a] > b->ndof[c]; });
  std::vector<std::vector<int>> parts(G);
  std::vector<long long> load(G, 0);
  for (int i : order) {
    const int k = (int)(std::min_element(load.begin(), load.end()) - load.begin());
    parts[k].push_back(i);
    load[k] += b->ndof[i];
  }
  for (auto& p : parts) std::sort(p.begin(), p.end());
  parts.erase(std::remove_if(parts.begin(), parts.end(), [](const std::vector<int>& p) { return p.empty(); }),
              parts.end());
  return parts;
}

void gather(BGroup* g) {
  const int n = (int)g->idx.size();
  dd::launch_b_gather(g->B, n, g->stat_d, g->s);
  DD_CUDA(cudaMemcpyAsync(g->stat_h, g->stat_d, sizeof(BStat) * n, cudaMemcpyDeviceToHost, g->s));
  DD_CUDA(cudaStreamSynchronize(g->s));
}

// images of the outer step (as the plain one): b = M w (w2), x = w / ||w||_M (xe), A_sigma x
// with x^T A_sigma x, and the residual norms
void outer_images(BGroup* g, int w_role) {
  dd::launch_b_stencil(g->B, g->vm_st, g->n_st, 1, w_role, dd::BV_W2, g->s);
  dd::launch_b_outer_normalize(g->B, g->vm_vec, g->n_vec, w_role, dd::BV_W2, dd::BV_XE, g->s);
  dd::launch_b_stencil_dot(g->B, g->vm_sdot, g->n_sdot, dd::BV_XE, dd::BV_W3, g->s);
  dd::launch_b_outer_res(g->B, g->vm_vec, g->n_vec, dd::BV_W3, dd::BV_W2, g->s);
}

struct Outputs {
  double* lambda;
  int* outer;
  int* inner;
  double* seconds;
  std::chrono::steady_clock::time_point t0;
  double now() const { return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count(); }
};

// readiness of each instance's set-up: 0 running, 1 done, < 0 its failure status
using Ready = std::vector<std::atomic<int>>;

// Instances of the group whose set-up has completed since the last look (the caller starts
// them), or failed (moved to DONE with their status).
std::vector<int> take_ready(BGroup* g, const Ready& ready, std::vector<int>& state, std::vector<int>& status) {
  std::vector<int> fresh;
  for (size_t j = 0; j < g->idx.size(); ++j) {
    if (state[j] != ST_PENDING) continue;
    const int r = ready[g->idx[j]].load(std::memory_order_acquire);
    if (r == 1) {
      fresh.push_back((int)j);
    } else if (r < 0) {
      state[j] = ST_DONE;
      status[j] = r;
    }
  }
  return fresh;
}

int finish(BGroup* g, const std::vector<int>& status, const std::vector<double>& rho, const std::vector<int>& outer,
           const std::vector<int>& inner, const std::vector<double>& secs, const Outputs& o) {
  int herr = 0;
  DD_CUDA(cudaMemcpyAsync(&herr, g->err_d + 8, sizeof(int), cudaMemcpyDeviceToHost, g->s));
  DD_CUDA(cudaStreamSynchronize(g->s));
  int first = DD_OK;
  for (size_t j = 0; j < g->idx.size(); ++j) {
    const int i = g->idx[j];
    if (o.lambda) o.lambda[i] = rho[j];
    if (o.outer) o.outer[i] = outer[j];
    if (o.inner) o.inner[i] = inner[j];
    if (o.seconds) o.seconds[i] = secs[j];
    if (status[j] != DD_OK && first == DD_OK) first = status[j];
  }
  if (herr != 0) {
    DD_CUDA(cudaMemsetAsync(g->err_d + 8, 0, sizeof(int), g->s));
    DD_CUDA(cudaStreamSynchronize(g->s));
    return DD_ETIMEOUT;
  }
  return first;
}

// Batched shifted inverse iteration of one group (the stop rule and inner tolerance of
// dd_eigenpair): each instance joins when its set-up is done and runs the steps of
// dd_inverse_iterate; one outer step of every running instance per pass.
int run_ipm(dd_batch* b, BGroup* g, const Ready& ready, const Outputs& o) {
  using namespace dd;
  const int m = (int)g->idx.size();
  const double tol_res = 1e-8, tol_lam = 1e-10, rtol_inner = 1e-8;
  const int maxit_outer = 100, maxit_inner = 10000;
  std::vector<int> state(m, ST_PENDING), outer(m, 0), inner(m, 0), status(m, DD_OK);
  std::vector<double> rho(m, 0.0), rho_prev(m, 0.0), secs(m, 0.0);
  for (int j = 0; j < m; ++j) g->Bh[j].r = b->ctx[g->idx[j]]->r;
  mask(g, [](int) { return false; });
  launch_b_mark_done(g->B, m, g->s);   // the contraction's tiles skip instances not yet joined
  while (true) {
    const std::vector<int> fresh = take_ready(g, ready, state, status);
    if (!fresh.empty()) {
      // x_0 -> M-normalised iterate and its images, the newcomers only
      for (int j : fresh) DD_CUDA(cudaMemsetAsync(b->ctx[g->idx[j]]->ost, 0, sizeof(OuterState), g->s));
      std::vector<char> on(m, 0);
      for (int j : fresh) on[j] = 1;
      mask(g, [&](int j) { return on[j] != 0; });
      launch_b_pad(g->B, g->vm_vec, g->n_vec, g->xptr_d, BV_W1, g->s);
      outer_images(g, BV_W1);
      gather(g);
      for (int j : fresh) {
        if (g->stat_h[j].outer_status != 0) {
          state[j] = ST_DONE;
          status[j] = g->stat_h[j].outer_status;
          secs[j] = o.now();
          continue;
        }
        rho_prev[j] = rho[j] = b->ctx[g->idx[j]]->sigma + g->stat_h[j].xAx;
        state[j] = ST_RUNNING;
      }
    }
    int running = 0, pending = 0;
    for (int j = 0; j < m; ++j) {
      running += state[j] == ST_RUNNING;
      pending += state[j] == ST_PENDING;
    }
    if (running == 0) {
      if (pending == 0) break;
      std::this_thread::sleep_for(std::chrono::microseconds(20));
      continue;
    }
    // A_sigma w = M x_k by PCG from zero, every running instance
    mask(g, [&](int j) { return state[j] == ST_RUNNING; });
    launch_b_zero_pcg(g->B, g->vm_vec, g->n_vec, g->s);
    launch_b_pcg_reset(g->B, m, rtol_inner * rtol_inner, maxit_inner, g->s);
    launch_b_pcg_init(g->B, g->vm_init, g->n_init, BV_W2, g->s);
    precond(g, 1);
    for (int it = 0; it < maxit_inner + g->check_every; it += g->check_every) {
      DD_CUDA(cudaGraphLaunch(g->graph, g->s));
      note_launches(g->graph_kernels);
      gather(g);
      bool all = true;
      for (int j = 0; j < m; ++j)
        if (state[j] == ST_RUNNING && !g->stat_h[j].pcg_done) all = false;
      if (all) break;
    }
    for (int j = 0; j < m; ++j) {
      if (state[j] != ST_RUNNING) continue;
      inner[j] += g->stat_h[j].pcg_iter;
      const int ps = g->stat_h[j].pcg_status;
      if (ps != 0 && ps != DD_EMAXIT) {
        state[j] = ST_DONE;
        status[j] = ps;
        outer[j] += 1;
        secs[j] = o.now();
      }
    }
    mask(g, [&](int j) { return state[j] == ST_RUNNING; });
    outer_images(g, BV_X);
    gather(g);
    const double now = o.now();
    for (int j = 0; j < m; ++j) {
      if (state[j] != ST_RUNNING) continue;
      const BStat& h = g->stat_h[j];
      outer[j] += 1;
      if (h.outer_status != 0) {
        state[j] = ST_DONE;
        status[j] = h.outer_status;
        secs[j] = now;
        continue;
      }
      rho[j] = b->ctx[g->idx[j]]->sigma + h.xAx;
      const double eta = std::sqrt(h.rr / h.mm) / std::fabs(rho[j]);
      if (!std::isfinite(rho[j])) {
        state[j] = ST_DONE;
        status[j] = DD_ENAN;
        secs[j] = now;
      } else if (eta <= tol_res && std::fabs(rho[j] - rho_prev[j]) <= tol_lam * std::fabs(rho[j])) {
        state[j] = ST_DONE;
        secs[j] = now;
      } else if (outer[j] >= maxit_outer) {
        state[j] = ST_DONE;
        status[j] = DD_EMAXIT;
        secs[j] = now;
      } else {
        rho_prev[j] = rho[j];
      }
    }
  }
  // phi (the M-normalised iterate) back to the instances' vectors
  mask(g, [&](int) { return true; });
  launch_b_unpad_active(g->B, g->vm_vec, g->n_vec, BV_XE, g->xptr_d, g->s);
  return finish(g, status, rho, outer, inner, secs, o);
}

// Batched SI-LOPCG with the fused inner step (Algorithm 1 with w_k = M_AS2^{-1} r_o, Sec. 4.3)
// of one group: the steps of dd_lopcg for every running instance at once.  The twelve work
// vectors play the same roles in every instance (the roles rotate in lockstep; a newcomer
// starts in the current roles, all of them initialised), so each launch names roles.
int run_lopcg_fused(dd_batch* b, BGroup* g, const Ready& ready, const Outputs& o) {
  using namespace dd;
  const int m = (int)g->idx.size();
  const double tol_res = 1e-8, tol_lam = 1e-10;
  const int maxit_outer = 1000;
  for (int j = 0; j < m; ++j) {
    dd_ctx* c = b->ctx[g->idx[j]];
    BInst& I = g->Bh[j];
    for (int k = 0; k < 12; ++k) I.lop[k] = c->lop[k];
    I.lst = c->lst;
    I.lop_red = c->lop_red;
    I.r = c->lop[9];   // the preconditioner is applied to the outer residual r_o
  }
  mask(g, [](int) { return false; });
  launch_b_mark_done(g->B, m, g->s);
  int X = 0, XP = 1, T = 2, AX = 3, AXP = 4, MX = 5, MXP = 6;
  const int AW = 7, MW = 8, RO = 9;
  int AT = 10, MT = 11;
  auto R = [](int k) { return BV_LOP + k; };
  cudaStream_t s = g->s;
  const long long first = (long long)g->ypad;   // the first interior node (p = 1)
  std::vector<int> state(m, ST_PENDING), outer(m, 0), inner(m, 0), status(m, DD_OK), exact(m, 1), xrole(m, 0);
  std::vector<double> lam(m, 0.0), rr(m, 0.0), mm(m, 0.0), rho(m, 0.0), secs(m, 0.0);
  std::vector<double> rho_prev(m, std::numeric_limits<double>::infinity());
  auto explicit_images = [&]() {
    launch_b_stencil_role(g->B, g->vm_st, g->n_st, 1, R(X), R(MX), s);
    launch_b_lop_normalize(g->B, g->vm_vec, g->n_vec, R(X), R(MX), s);
    launch_b_stencil_dot(g->B, g->vm_sdot, g->n_sdot, R(X), R(AX), s);
    launch_b_outer_res_ro(g->B, g->vm_vec, g->n_vec, R(AX), R(MX), R(RO), s);
    gather(g);
  };
  auto stops = [&](double rh, double r2, double m2, double prev) {
    const double eta = std::sqrt(r2 / m2) / std::fabs(rh);
    return eta <= tol_res && std::fabs(rh - prev) <= tol_lam * std::fabs(rh);
  };
  auto done = [&](int j, int st) {
    state[j] = ST_DONE;
    status[j] = st;
    xrole[j] = X;
    secs[j] = o.now();
  };
  while (true) {
    const std::vector<int> fresh = take_ready(g, ready, state, status);
    if (!fresh.empty()) {
      // x_0 = e_1 and x_1 = the instance's vector, M-normalised, with their images
      std::vector<char> on(m, 0);
      for (int j : fresh) on[j] = 1;
      mask(g, [&](int j) { return on[j] != 0; });
      launch_b_zero_roles(g->B, g->vm_vec, g->n_vec, BV_LOP, 12, s);
      launch_b_lop_reset(g->B, m, s);
      launch_b_set_entry(g->B, m, R(XP), first, 1.0, s);
      launch_b_stencil_role(g->B, g->vm_st, g->n_st, 1, R(XP), R(MXP), s);
      launch_b_lop_normalize(g->B, g->vm_vec, g->n_vec, R(XP), R(MXP), s);
      launch_b_stencil_role(g->B, g->vm_st, g->n_st, 0, R(XP), R(AXP), s);
      launch_b_pad(g->B, g->vm_vec, g->n_vec, g->xptr_d, R(X), s);
      explicit_images();
      for (int j : fresh) {
        if (g->stat_h[j].outer_status != 0) {
          done(j, g->stat_h[j].outer_status);
          continue;
        }
        lam[j] = g->stat_h[j].xAx;
        rr[j] = g->stat_h[j].rr;
        mm[j] = g->stat_h[j].mm;
        exact[j] = 1;
        state[j] = ST_RUNNING;
      }
    }
    // stop test; instances whose images are carried combinations confirm on recomputed ones
    std::vector<int> confirm;
    for (int j = 0; j < m; ++j) {
      if (state[j] != ST_RUNNING) continue;
      rho[j] = b->ctx[g->idx[j]]->sigma + lam[j];
      if (!std::isfinite(rho[j])) {
        done(j, DD_ENAN);
        continue;
      }
      if (stops(rho[j], rr[j], mm[j], rho_prev[j])) {
        if (exact[j]) done(j, DD_OK);
        else confirm.push_back(j);
      }
    }
    if (!confirm.empty()) {
      std::vector<char> on(m, 0);
      for (int j : confirm) on[j] = 1;
      mask(g, [&](int j) { return on[j] != 0; });
      explicit_images();
      for (int j : confirm) {
        exact[j] = 1;
        lam[j] = g->stat_h[j].xAx;
        rr[j] = g->stat_h[j].rr;
        mm[j] = g->stat_h[j].mm;
        const double rho_e = b->ctx[g->idx[j]]->sigma + lam[j];
        if (stops(rho_e, rr[j], mm[j], rho_prev[j])) {
          rho[j] = rho_e;
          done(j, DD_OK);
        }
      }
    }
    for (int j = 0; j < m; ++j)
      if (state[j] == ST_RUNNING && outer[j] >= maxit_outer) done(j, DD_EMAXIT);
    int running = 0, pending = 0;
    for (int j = 0; j < m; ++j) {
      running += state[j] == ST_RUNNING;
      pending += state[j] == ST_PENDING;
    }
    if (running == 0) {
      if (pending == 0) break;
      std::this_thread::sleep_for(std::chrono::microseconds(20));
      continue;
    }
    // w = M_AS2^{-1} r_o; images of w; Rayleigh-Ritz on span{x_k, w, x_{k-1}}; update
    mask(g, [&](int j) { return state[j] == ST_RUNNING; });
    launch_b_pcg_reset(g->B, m, 0.0, 0, s);
    precond(g, 0);
    launch_b_stencil2(g->B, g->vm_st2, g->n_st2, BV_Z, R(AW), R(MW), s);
    const int S[3] = {R(X), BV_Z, R(XP)}, AS[3] = {R(AX), R(AW), R(AXP)}, MS[3] = {R(MX), R(MW), R(MXP)};
    launch_b_lop_gram(g->B, g->vm_vec, g->n_vec, S, AS, MS, 1e-10, s);
    launch_b_lop_update3(g->B, g->vm_vec, g->n_vec, S, AS, MS, R(T), R(AT), R(MT), R(RO), s);
    int t0 = XP;
    XP = X; X = T; T = t0;
    t0 = AXP; AXP = AX; AX = AT; AT = t0;
    t0 = MXP; MXP = MX; MX = MT; MT = t0;
    gather(g);
    for (int j = 0; j < m; ++j) {
      if (state[j] != ST_RUNNING) continue;
      inner[j] += 1;
      outer[j] += 1;
      if (g->stat_h[j].lop_status != 0) {
        done(j, g->stat_h[j].lop_status);
        continue;
      }
      rho_prev[j] = rho[j];
      lam[j] = g->stat_h[j].theta;
      rr[j] = g->stat_h[j].lop_rr;
      mm[j] = g->stat_h[j].lop_mm;
      exact[j] = 0;
    }
  }
  // phi back to the instances' vectors, each from the role its iterate had when it stopped
  for (int role = 0; role < 12; ++role) {
    bool any = false;
    for (int j = 0; j < m; ++j) any = any || (state[j] == ST_DONE && xrole[j] == role);
    if (!any) continue;
    mask(g, [&](int j) { return xrole[j] == role; });
    launch_b_unpad_active(g->B, g->vm_vec, g->n_vec, R(role), g->xptr_d, s);
  }
  for (int j = 0; j < m; ++j) g->Bh[j].r = b->ctx[g->idx[j]]->r;
  upload(g);
  return finish(g, status, rho, outer, inner, secs, o);
}

const int kGroupChoices[] = {1, 2, 4, 8};

// the group count of this call: fixed, or the next one not yet timed for this method, or the
// fastest timed (every count gives the same results, so this only moves the speed)
int choose_groups(const dd_batch* b, int method) {
  const int n = (int)b->ctx.size();
  if (b->groups_opt > 0) return std::min(b->groups_opt, n);
  int best = 1;
  double best_t = std::numeric_limits<double>::infinity();
  for (int G : kGroupChoices) {
    if (G > n) break;
    auto it = b->timed.find((long long)method * 1000 + G);
    if (it == b->timed.end()) return G;
    if (it->second < best_t) {
      best_t = it->second;
      best = G;
    }
  }
  return best;
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
    if (cudaMemset(b->Ainv_all, 0, ba) != cudaSuccess || cudaMemset(b->Rpack_all, 0, br) != cudaSuccess ||
        cudaMemset(b->Y_all, 0, by) != cudaSuccess) {
      cudaGetLastError();
      destroy_all(b);
      return DD_ECUDA;
    }
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

int dd_batch_set_groups(dd_batch* b, int groups) {
  if (!b || groups < -1) return DD_EINVAL;
  b->groups_opt = groups;
  return DD_OK;
}

int dd_batch_info(const dd_batch* b, int* batchable_out, int* last_batched_out, int* gemm_tile_n_out,
                  int* groups_out, double* setup_seconds_out, double* total_seconds_out) {
  if (!b) return DD_EINVAL;
  if (batchable_out) *batchable_out = b->eligible ? 1 : 0;
  if (last_batched_out) *last_batched_out = b->last_batched;
  if (gemm_tile_n_out) *gemm_tile_n_out = b->last_bn;
  if (groups_out) *groups_out = b->last_groups;
  if (setup_seconds_out) *setup_seconds_out = b->last_setup_s;
  if (total_seconds_out) *total_seconds_out = b->last_total_s;
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
  if (threads < 1) threads = std::min(n, 16);
  threads = std::min(threads, n);
  b->last_batched = 0;
  // the batched kernels need the options they were built for (the fused p update, the grouped
  // contraction and the cyclic-reduction coarse solve, PCG inner solves)
  bool engine = b->eligible && b->groups_opt >= 0 && (method == DD_BATCH_IPM || method == DD_BATCH_LOPCG_FUSED);
  for (dd_ctx* c : b->ctx)
    if (c->krylov != 0 || c->ras != 0 || c->coarse_mode == 2 || c->timing || c->fused_pq_opt == 0 ||
        c->pq_pairs != b->ctx.front()->pq_pairs || c->fuse_xr != b->ctx.front()->fuse_xr)
      engine = false;
  const auto t_start = std::chrono::steady_clock::now();
  std::vector<double> setup_s(n, 0.0);
  Ready ready(n);
  for (auto& r : ready) r.store(0);
  int G = 0;
  bool fresh_engine = false;
  if (engine) {
    try {
      DD_CUDA(cudaSetDevice(b->device));
      if (method == DD_BATCH_LOPCG_FUSED) ensure_lopcg(b);   // before any worker touches a context
    } catch (const dd::Error& e) {
      return e.code;
    }
    const long long sig = option_signature(b);
    if (sig != b->opt_sig) {
      drop_engines(b);
      b->opt_sig = sig;
    }
    G = choose_groups(b, method);
    fresh_engine = b->engines.find(G) == b->engines.end();
  }
  std::vector<int> order(n);
  for (int i = 0; i < n; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](int a, int c) { return b->ndof[a] > b->ndof[c]; });
  std::atomic<int> next{0};
  std::atomic<int> first_error{DD_OK};
  auto note_error = [&](int rc) {
    int expect = DD_OK;
    first_error.compare_exchange_strong(expect, rc);
  };
  auto worker = [&]() {
    cudaSetDevice(b->device);
    cudaStream_t s = nullptr;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) {
      cudaGetLastError();
      note_error(DD_ECUDA);
      for (int k = next.fetch_add(1); k < n; k = next.fetch_add(1)) ready[order[k]].store(DD_ECUDA);
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
      ready[i].store(rc == DD_OK ? 1 : rc, std::memory_order_release);
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
      if (rc != DD_OK) note_error(rc);
    }
    cudaStreamDestroy(s);
  };
  std::vector<std::thread> pool;
  pool.reserve(threads);
  for (int t = 0; t < threads; ++t) pool.emplace_back(worker);
  int rc = DD_OK;
  if (engine) {
    // a group count used for the first time is built once every instance is set up (its
    // contraction tile is timed on the instances' operands); later calls let each instance
    // join its group's iteration as soon as its own set-up is done
    if (fresh_engine) {
      for (auto& th : pool) th.join();
      pool.clear();
      rc = first_error.load();
      if (rc == DD_OK) {
        std::vector<BGroup*> gs;
        try {
          for (const auto& part : partition(b, G)) gs.push_back(build_group(b, part));
          b->engines[G] = gs;
        } catch (const dd::Error& e) {
          for (BGroup* g : gs) free_group(g);
          rc = e.code;
        }
      }
    }
    if (rc == DD_OK) {
      std::vector<BGroup*>& gs = b->engines[G];
      const Outputs o{lambda_out, outer_out, inner_out, seconds_out, t_start};
      std::vector<int> grc(gs.size(), DD_OK);
      std::vector<std::thread> gthreads;
      for (size_t k = 0; k < gs.size(); ++k)
        gthreads.emplace_back([&, k]() {
          try {
            DD_CUDA(cudaSetDevice(b->device));
            grc[k] = method == DD_BATCH_IPM ? run_ipm(b, gs[k], ready, o) : run_lopcg_fused(b, gs[k], ready, o);
          } catch (const dd::Error& e) {
            grc[k] = e.code;
          } catch (...) {
            grc[k] = DD_ECUDA;
          }
        });
      for (auto& th : gthreads) th.join();
      for (int r : grc)
        if (r != DD_OK && rc == DD_OK) rc = r;
      b->last_batched = 1;
      b->last_groups = (int)gs.size();
      b->last_bn = gs.front()->bn;
    }
  }
  for (auto& th : pool) th.join();
  if (rc == DD_OK) rc = first_error.load();
  if (rc == DD_OK && engine) {
    // bounded waits of the instances' coarse solves
    for (dd_ctx* c : b->ctx) {
      int e = 0;
      if (cudaMemcpy(&e, c->dev_err + 8, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) {
        cudaGetLastError();
        rc = DD_ECUDA;
        break;
      }
      if (e != 0) {
        cudaMemset(c->dev_err + 8, 0, sizeof(int));
        rc = DD_ETIMEOUT;
      }
    }
  }
  b->last_setup_s = 0.0;
  for (double t : setup_s) b->last_setup_s = std::max(b->last_setup_s, t);
  b->last_total_s = std::chrono::duration<double>(std::chrono::steady_clock::now() - t_start).count();
  if (rc == DD_OK && engine && !fresh_engine) {
    double& t = b->timed.emplace((long long)method * 1000 + G, b->last_total_s).first->second;
    t = std::min(t, b->last_total_s);
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
