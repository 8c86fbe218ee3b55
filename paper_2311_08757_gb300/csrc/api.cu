// C ABI and host runtime: context set-up, the PCG engine (eager launches or a replayed
// CUDA graph of a block of iterations), the shifted inverse iteration, staging of host
// buffers, error reporting.
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <limits>
#include <utility>
#include <new>

#include "dd_band.cuh"

using dd::Error;

namespace {

thread_local std::string g_setup_err;

bool is_device_ptr(const void* p) {
  if (p == nullptr) return false;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

int fail(dd_ctx* c, int code, const std::string& msg) {
  if (c) c->err = msg;
  else g_setup_err = msg;
  return code;
}

template <typename F>
int guarded(dd_ctx* c, F&& f) {
  try {
    const int rc = f();
    // a bounded device wait that expired (tensor-core GEMM pipeline, coarse-solve copy) left
    // its bit in the error word; the results of that call cannot be trusted
    if (rc == DD_OK && c != nullptr && c->dev_err != nullptr) {
      int e = 0;
      DD_CUDA(cudaMemcpyAsync(&e, c->dev_err + 8, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
      DD_CUDA(cudaStreamSynchronize(c->stream));
      if (e != 0) {
        DD_CUDA(cudaMemsetAsync(c->dev_err + 8, 0, sizeof(int), c->stream));
        return fail(c, DD_ETIMEOUT, "a bounded device wait expired (code " + std::to_string(e) + ")");
      }
    }
    return rc;
  } catch (const Error& e) {
    return fail(c, e.code, e.msg);
  } catch (const std::bad_alloc&) {
    return fail(c, DD_ENOMEM, "host allocation failed");
  } catch (...) {
    return fail(c, DD_ECUDA, "unexpected exception");
  }
}

}  // namespace

namespace dd {

// Padded box vector with a zeroed guard band of kVecGuard doubles on each side: the
// 3^d-point stencil of the first (last) interior node reaches one element before (after)
// the padded range, where the homogeneous Dirichlet value 0 must be read.
constexpr long long kVecGuard = 64;   // 512 bytes, keeps the 256-byte alignment
double* alloc_vec(dd_ctx* c) {
  double* base = (double*)dev_alloc(c, sizeof(double) * (size_t)(c->g.plen + 2 * kVecGuard));
  return base + kVecGuard;
}

static std::atomic<long long> g_launches{0};
// launches issued while this thread captures a stream into a graph do not run: the graph's
// kernel nodes are counted when the graph is launched
static thread_local int t_capturing = 0;
void note_launch() {
  if (!t_capturing) g_launches.fetch_add(1, std::memory_order_relaxed);
}
void note_launches(long long k) { g_launches.fetch_add(k, std::memory_order_relaxed); }
long long launch_count() { return g_launches.load(std::memory_order_relaxed); }
void set_capturing(bool on) { t_capturing = on ? 1 : 0; }
long long graph_kernel_nodes(cudaGraph_t gr) {
  size_t n = 0;
  DD_CUDA(cudaGraphGetNodes(gr, nullptr, &n));
  std::vector<cudaGraphNode_t> nodes(n);
  if (n) DD_CUDA(cudaGraphGetNodes(gr, nodes.data(), &n));
  long long k = 0;
  for (size_t i = 0; i < n; ++i) {
    cudaGraphNodeType t;
    DD_CUDA(cudaGraphNodeGetType(nodes[i], &t));
    if (t == cudaGraphNodeTypeKernel) ++k;
  }
  return k;
}

void* dev_alloc(dd_ctx* c, size_t bytes) {
  void* p = nullptr;
  if (bytes == 0) bytes = 16;
  cudaError_t e = cudaMalloc(&p, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    throw Error(DD_ENOMEM, std::string("cudaMalloc(") + std::to_string(bytes) + "): " + cudaGetErrorString(e));
  }
  DD_CUDA(cudaMemsetAsync(p, 0, bytes, c->stream));
  c->allocs.push_back(p);
  c->bytes += (long long)bytes;
  return p;
}

static const char* kClassNames[KC_COUNT] = {
    "stencil_Asigma", "p_update", "xr_update", "local_solve_fp64", "pack_restrict", "local_gemm_tc",
    "prolong_sum", "coarse_restrict", "coarse_solve", "outer_step", "misc", "rayleigh_ritz", "pack_xr_update"};

void timer_begin(dd_ctx* c, int, cudaStream_t s, cudaEvent_t* e0) {
  *e0 = nullptr;
  if (!c->timing) return;
  DD_CUDA(cudaEventCreate(e0));
  DD_CUDA(cudaEventRecord(*e0, s));
}

void timer_end(dd_ctx* c, int kc, cudaStream_t s, cudaEvent_t e0) {
  if (!c->timing || e0 == nullptr) return;
  cudaEvent_t e1;
  DD_CUDA(cudaEventCreate(&e1));
  DD_CUDA(cudaEventRecord(e1, s));
  c->timer.pending.push_back({kc, {e0, e1}});
}

void timer_collect(dd_ctx* c) {
  for (auto& pe : c->timer.pending) {
    float ms = 0.f;
    DD_CUDA(cudaEventSynchronize(pe.second.second));
    DD_CUDA(cudaEventElapsedTime(&ms, pe.second.first, pe.second.second));
    c->timer.ms[pe.first] += ms;
    c->timer.launches[pe.first] += 1;
    cudaEventDestroy(pe.second.first);
    cudaEventDestroy(pe.second.second);
  }
  c->timer.pending.clear();
}

}  // namespace dd

#define TIMED(kc, stream, body)            \
  do {                                     \
    cudaEvent_t e0_;                       \
    dd::timer_begin(c, kc, stream, &e0_);  \
    body;                                  \
    dd::timer_end(c, kc, stream, e0_);     \
  } while (0)

namespace {

using namespace dd;

// FP64 local solves: groups of up to k consecutive slots of one type, one group per warp
void set_local_groups(dd_ctx* c, int k) {
  c->rhs_k = k;
  c->group_h.clear();
  for (int t = 0; t < c->ntypes; ++t)
    for (int j = 0; j < c->type_count[t]; j += k)
      c->group_h.push_back(make_int2(c->type_first[t] + j, std::min(k, c->type_count[t] - j)));
  c->ngroups = (int)c->group_h.size();
  DD_CUDA(cudaMemcpyAsync(c->groups, c->group_h.data(), sizeof(int2) * c->group_h.size(), cudaMemcpyHostToDevice,
                          c->stream));
}

void build_subdomains(dd_ctx* c) {
  const Geo& g = c->g;
  int id_of[16];
  for (int k = 0; k < 16; ++k) id_of[k] = -1;
  c->ntypes = 0;
  c->subs_h.resize(g.nsub);
  const int L2 = (g.p == 2) ? g.L : 1;
  for (int s = 0; s < g.nsub; ++s) {
    const int i1 = (g.p == 1) ? s : s / g.L, i2 = (g.p == 1) ? 0 : s % g.L;
    const int t1 = ax_type(g, i1), t2 = (g.p == 2) ? ax_type(g, i2) : 0;
    const int key = t1 * 4 + t2;
    if (id_of[key] < 0) {
      id_of[key] = c->ntypes;
      c->type_ax[c->ntypes][0] = t1;
      c->type_ax[c->ntypes][1] = t2;
      ++c->ntypes;
    }
    Sub sb;
    sb.type = id_of[key];
    sb.lo1 = ax_lo(g, i1);
    sb.w1 = ax_hi(g, i1) - sb.lo1 + 1;
    if (g.p == 2) {
      sb.lo2 = ax_lo(g, i2);
      sb.w2 = ax_hi(g, i2) - sb.lo2 + 1;
    } else {
      sb.lo2 = 0;
      sb.w2 = 1;
    }
    sb.nloc = sb.w1 * sb.w2 * g.nyi;
    c->subs_h[s] = sb;
    c->type_nloc[sb.type] = sb.nloc;
    c->type_w1[sb.type] = sb.w1;
    c->type_w2[sb.type] = sb.w2;
  }
  (void)L2;
  c->type_count.assign(c->ntypes, 0);
  for (const Sub& s : c->subs_h) c->type_count[s.type]++;
  c->type_first.assign(c->ntypes, 0);
  for (int t = 1; t < c->ntypes; ++t) c->type_first[t] = c->type_first[t - 1] + c->type_count[t - 1];
  std::vector<int> next = c->type_first, slot(g.nsub);
  for (int s = 0; s < g.nsub; ++s) slot[s] = next[c->subs_h[s].type]++;
  c->nloc_max = 0;
  int w2max = 1, nlp_max = 0;
  for (int t = 0; t < c->ntypes; ++t) {
    c->nloc_max = std::max(c->nloc_max, c->type_nloc[t]);
    w2max = std::max(w2max, c->type_w2[t]);
    nlp_max = std::max(nlp_max, c->type_nloc[t] / g.nyi * g.Ypad);   // columns x Ypad slots
  }
  // K of the local contraction: whole 128-byte swizzle rows of the operand type (64 BF16,
  // 32 TF32, 128 E4M3 values), over the column-padded local length
  const int kq = c->grid.precision == DD_PREC_FP8 ? 128 : 64;
  c->kpad = (nlp_max + kq - 1) / kq * kq;
  c->band = (g.p == 1) ? g.nyi + 1 : w2max * g.nyi + g.nyi + 1;
  c->subs = (Sub*)dev_alloc(c, sizeof(Sub) * g.nsub);
  c->slot_of_sub = (int*)dev_alloc(c, sizeof(int) * g.nsub);
  // index tables of the prolong-sum: owners of every x node column, row offsets per subdomain
  std::vector<int4> ax(g.ncx), sr(g.nsub);
  for (int a = 0; a < g.ncx; ++a) {
    int4 v = make_int4(-1, 0, -1, 0);
    int k = 0;
    // subdomain i spans columns i n - delta + 1 .. (i + 1) n + delta - 1 (clipped), so only
    // i = floor(a / n) - 1 .. floor(a / n) + 1 can hold column a (2 delta < n); scanned in
    // increasing i, the order the owners are listed in
    const int i0 = std::max(0, a / g.n - 1), i1 = std::min(g.L - 1, a / g.n + 1);
    for (int i = i0; i <= i1 && k < 2; ++i)
      if (a >= ax_lo(g, i) && a <= ax_hi(g, i)) {
        if (k == 0) { v.x = i; v.y = a - ax_lo(g, i); }
        else { v.z = i; v.w = a - ax_lo(g, i); }
        ++k;
      }
    ax[a] = v;
  }
  for (int s = 0; s < g.nsub; ++s)
    sr[s] = make_int4(slot[s] * c->kpad, c->subs_h[s].type * c->kpad, c->subs_h[s].w2, c->subs_h[s].nloc);
  std::vector<int> sos(g.nsub);
  for (int s2 = 0; s2 < g.nsub; ++s2) sos[slot[s2]] = s2;
  c->sub_of_slot = (int*)dev_alloc(c, sizeof(int) * g.nsub);
  c->groups = (int2*)dev_alloc(c, sizeof(int2) * g.nsub);
  DD_CUDA(cudaMemcpyAsync(c->sub_of_slot, sos.data(), sizeof(int) * g.nsub, cudaMemcpyHostToDevice, c->stream));
  set_local_groups(c, std::min(2, rhs_per_warp(c->nloc_max, c->band)));
  // p = 1: the prolong-sum computes owners and packed rows in closed form where the formula
  // reproduces these tables exactly (every column, packed row i = subdomain i)
  bool closed = g.p == 1;
  for (int a = 1; closed && a <= g.nxi; ++a) {
    const int4 v = p1_owners(g, a), t = ax[a];
    closed = v.x == t.x && v.y == t.y && v.z == t.z && (t.z < 0 || v.w == t.w);
  }
  for (int s2 = 0; closed && s2 < g.nsub; ++s2) closed = slot[s2] == s2;
  if (g.p == 1) {
    c->ptypes = make_int4(c->subs_h[0].type, g.L >= 3 ? c->subs_h[1].type : 0, c->subs_h[g.L - 1].type, 0);
    for (int s2 = 0; closed && s2 < g.nsub; ++s2) {
      const int want = s2 == 0 ? c->ptypes.x : (s2 == g.L - 1 ? c->ptypes.z : c->ptypes.y);
      closed = c->subs_h[s2].type == want;
    }
  }
  c->prolong_closed = closed ? 1 : 0;
  c->prolong_arith = (closed && !c->prolong_tables_opt) ? 1 : 0;
  c->axown = (int4*)dev_alloc(c, sizeof(int4) * g.ncx);
  c->subrow = (int4*)dev_alloc(c, sizeof(int4) * g.nsub);
  DD_CUDA(cudaMemcpyAsync(c->axown, ax.data(), sizeof(int4) * g.ncx, cudaMemcpyHostToDevice, c->stream));
  DD_CUDA(cudaMemcpyAsync(c->subrow, sr.data(), sizeof(int4) * g.nsub, cudaMemcpyHostToDevice, c->stream));
  if (g.p == 1) {
    // per node column a and owner: its packed row and type row advanced to the column's local
    // position; an absent owner repeats subdomain 0's rows (a valid address, masked)
    std::vector<int4> crw(g.ncx);
    for (int a = 0; a < g.ncx; ++a) {
      const int4 t = ax[a];
      const int o0 = t.x >= 0 ? t.x : 0, o1 = t.z >= 0 ? t.z : 0;
      const int l0 = t.x >= 0 ? t.y : 0, l1 = t.z >= 0 ? t.w : 0;
      crw[a] = make_int4(sr[o0].x + l0 * g.Ypad, sr[o0].y + l0 * g.Ypad, sr[o1].x + l1 * g.Ypad, sr[o1].y + l1 * g.Ypad);
    }
    c->colrow = (int4*)dev_alloc(c, sizeof(int4) * g.ncx);
    DD_CUDA(cudaMemcpyAsync(c->colrow, crw.data(), sizeof(int4) * g.ncx, cudaMemcpyHostToDevice, c->stream));
  }
  DD_CUDA(cudaMemcpyAsync(c->subs, c->subs_h.data(), sizeof(Sub) * g.nsub, cudaMemcpyHostToDevice, c->stream));
  DD_CUDA(cudaMemcpyAsync(c->slot_of_sub, slot.data(), sizeof(int) * g.nsub, cudaMemcpyHostToDevice, c->stream));
  DD_CUDA(cudaStreamSynchronize(c->stream));
}


// user vector (ABI order, host or device) -> padded device vector
void load_vec(dd_ctx* c, const double* u, double* padded) {
  const Geo& g = c->g;
  const double* src = u;
  if (!is_device_ptr(u)) {
    DD_CUDA(cudaMemcpyAsync(c->stage_a, u, sizeof(double) * g.ndof, cudaMemcpyHostToDevice, c->stream));
    src = c->stage_a;
  }
  launch_pad(c, src, padded, c->stream);
}

void store_vec(dd_ctx* c, const double* padded, double* u) {
  const Geo& g = c->g;
  if (is_device_ptr(u)) {
    launch_unpad(c, padded, u, c->stream);
  } else {
    launch_unpad(c, padded, c->stage_b, c->stream);
    DD_CUDA(cudaMemcpyAsync(u, c->stage_b, sizeof(double) * g.ndof, cudaMemcpyDeviceToHost, c->stream));
  }
}

// order the context's private stream after everything already queued on the caller's stream
void enter(dd_ctx* c) {
  DD_CUDA(cudaEventRecord(c->ev_enter, c->user_stream));
  DD_CUDA(cudaStreamWaitEvent(c->stream, c->ev_enter, 0));
}

int stage_err(dd_ctx* c, int need) {
  if (c == nullptr) return DD_EINVAL;
  if (c->stage < need) return fail(c, DD_ESTATE, "call out of order");
  return DD_OK;
}

bool use_gemm(const dd_ctx* c) { return c->grid.precision != DD_PREC_FP64; }

// z = M^{-1} r on device padded vectors; mode 0 standalone, 1 PCG start, 2 PCG iteration.
// The coarse right-hand side is formed in the pass that gathers R_i r (local solve or pack);
// with tensor-core local solves the coarse solve then runs on a second stream beside the
// GEMM (the two-level operator is additive, so the branches are independent).
// packed: the restrictions were packed by launch_pack_xr (a fused iteration), whose r update
// the prolong-sum then applies.
void precond(dd_ctx* c, const double* r, int mode, double* zout = nullptr, bool packed = false) {
  cudaStream_t s = c->stream;
  const bool coarse = c->grid.coarse != 0;
  double* c0 = coarse ? c->c0 : nullptr;
  if (use_gemm(c)) {
    if (!packed) TIMED(KC_PACK, s, launch_pack(c, r, c0, s));
    if (coarse) {
      DD_CUDA(cudaEventRecord(c->ev_fork, s));
      DD_CUDA(cudaStreamWaitEvent(c->side, c->ev_fork, 0));
      TIMED(KC_CSOLVE, c->side, launch_coarse_solve(c, c->side));
      DD_CUDA(cudaEventRecord(c->ev_join, c->side));
    }
    int rc;
    TIMED(KC_GEMM, s, rc = launch_gemm(c, s));
    if (rc != DD_OK) throw Error(rc, "local GEMM launch failed");
    if (coarse) DD_CUDA(cudaStreamWaitEvent(s, c->ev_join, 0));
  } else {
    TIMED(KC_LOCAL_FP64, s, launch_band_solve_local(c, r, c0, s));
    if (coarse) TIMED(KC_CSOLVE, s, launch_coarse_solve(c, s));
  }
  TIMED(KC_PROLONG, s, launch_prolong(c, mode, s, zout, packed));
}

// The x/r update runs inside the restriction packing (launch_pack_xr) for p = 1 boxes with
// BF16/TF32 local inverses and the fused p update, when the partial sums of (r, r) fit the
// reduction buffer (one per subdomain).
// The p = 1 float-pair pass stages whole node columns of at most blockDim rows.
bool pairs_possible(const dd_ctx* c) { return c->g.p == 2 || c->g.Ypad <= 256; }

bool fuse_xr_possible(const dd_ctx* c) {
  return c->g.p == 1 && (c->grid.precision == DD_PREC_BF16 || c->grid.precision == DD_PREC_TF32) &&
         c->fused_pq_opt != 0 && c->g.nsub <= kMaxRedBlocksHost;
}

void pcg_iteration(dd_ctx* c) {
  cudaStream_t s = c->stream;
  if (c->g.p == 1 && c->fused_pq_opt != 0) {   // fused, two nodes per thread unless option 1
    TIMED(KC_STENCIL, s, launch_fused_pq(c, s));
  } else if (c->g.p == 2 && c->pq_pairs) {
    TIMED(KC_PUPDATE, s, launch_pupdate_pairs(c, s));
    TIMED(KC_STENCIL, s, launch_matvec_pq_pairs(c, s));
  } else {
    TIMED(KC_PUPDATE, s, launch_pupdate(c, s));
    TIMED(KC_STENCIL, s, launch_matvec_pq(c, s));
  }
  if (c->fuse_xr) {
    TIMED(KC_PACK_XR, s, launch_pack_xr(c, s));
    precond(c, c->r, 2, nullptr, true);
  } else {
    TIMED(KC_XRUPDATE, s, launch_xr_update(c, s));
    precond(c, c->r, 2);
  }
}

void reset_graph(dd_ctx* c) {
  if (c->graph) {
    cudaGraphExecDestroy(c->graph);
    c->graph = nullptr;
  }
  c->graph_iters = 0;
}

void build_graph(dd_ctx* c) {
  reset_graph(c);
  cudaGraph_t gr;
  DD_CUDA(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
  set_capturing(true);
  try {
    for (int i = 0; i < c->check_every; ++i) pcg_iteration(c);
  } catch (...) {
    set_capturing(false);
    cudaStreamEndCapture(c->stream, &gr);
    cudaGetLastError();
    throw;
  }
  set_capturing(false);
  DD_CUDA(cudaStreamEndCapture(c->stream, &gr));
  // captured launches do not run; replays are counted when the graph is launched
  c->graph_kernels = graph_kernel_nodes(gr);
  DD_CUDA(cudaGraphInstantiate(&c->graph, gr, 0));
  DD_CUDA(cudaGraphDestroy(gr));
  c->graph_iters = c->check_every;
}

// PCG on the context's padded vectors: b (device padded), x holds the initial guess.
int pcg_run(dd_ctx* c, const double* b, double rtol, int maxit, int* iters, double* relres) {
  cudaStream_t s = c->stream;
  PcgState init;
  std::memset(&init, 0, sizeof(init));
  init.tol2 = rtol * rtol;
  init.maxit = maxit;
  init.flexible = (c->flexible_opt < 0) ? (use_gemm(c) ? 1 : 0) : c->flexible_opt;
  DD_CUDA(cudaMemcpyAsync(c->st, &init, sizeof(init), cudaMemcpyHostToDevice, s));
  DD_CUDA(cudaMemsetAsync(c->pb[0], 0, sizeof(double) * c->g.plen, s));
  DD_CUDA(cudaMemsetAsync(c->pb[1], 0, sizeof(double) * c->g.plen, s));
  TIMED(KC_MISC, s, launch_pcg_init(c, b, s));
  precond(c, c->r, 1);
  const bool graph = c->use_graph && !c->timing;
  if (graph && (c->graph == nullptr || c->graph_iters != c->check_every)) build_graph(c);
  for (int done_iters = 0; done_iters < maxit + c->check_every; done_iters += c->check_every) {
    if (graph) {
      DD_CUDA(cudaGraphLaunch(c->graph, s));
      note_launches(c->graph_kernels);
    } else {
      for (int i = 0; i < c->check_every; ++i) pcg_iteration(c);
    }
    DD_CUDA(cudaMemcpyAsync(c->st_h, c->st, sizeof(PcgState), cudaMemcpyDeviceToHost, s));
    DD_CUDA(cudaStreamSynchronize(s));
    if (c->timing) timer_collect(c);
    if (c->st_h->done) break;
  }
  if (x_lag_target(c) != nullptr) TIMED(KC_MISC, s, launch_x_final(c, s));
  const PcgState& h = *c->st_h;
  if (iters) *iters = h.iter;
  if (relres) *relres = (h.rr0 > 0.0) ? std::sqrt(h.rr / h.rr0) : 0.0;
  if (h.status != 0) {
    if (h.status == DD_EMAXIT) return fail(c, DD_EMAXIT, "PCG reached maxit");
    return fail(c, h.status, h.status == DD_ENOTSPD ? "p^T A_sigma p <= 0" : "non-finite PCG iterate");
  }
  if (!h.done) return fail(c, DD_EMAXIT, "PCG did not finish");
  return DD_OK;
}

// Right-preconditioned restarted (flexible) GMRES on A_sigma x = b, x in c->x (initial guess
// in, solution out); stop when the true residual is <= rtol ||b - A x_0||.
int gmres_run(dd_ctx* c, const double* b, double rtol, int maxit, int* iters, double* relres) {
  cudaStream_t s = c->stream;
  const Geo& g = c->g;
  const int m = c->gm_restart;
  const int ld = m + 1;
  if (c->gm_alloc != m) {
    if (c->gm_alloc != 0) throw Error(DD_ESTATE, "GMRES restart length cannot change after the first solve");
    c->gm_V.resize(m + 1);
    c->gm_Z.resize(m);
    for (auto& v : c->gm_V) v = alloc_vec(c);
    for (auto& v : c->gm_Z) v = alloc_vec(c);
    c->gm_W = alloc_vec(c);
    c->gm_Vptr = (double**)dev_alloc(c, sizeof(double*) * (m + 1));
    c->gm_Zptr = (double**)dev_alloc(c, sizeof(double*) * m);
    DD_CUDA(cudaMemcpyAsync(c->gm_Vptr, c->gm_V.data(), sizeof(double*) * (m + 1), cudaMemcpyHostToDevice, s));
    DD_CUDA(cudaMemcpyAsync(c->gm_Zptr, c->gm_Z.data(), sizeof(double*) * m, cudaMemcpyHostToDevice, s));
    c->gm_part = (double*)dev_alloc(c, sizeof(double) * (size_t)(m + 1) * 304);
    c->gm_h = (double*)dev_alloc(c, sizeof(double) * (2 * ld + 1));
    c->gm_H = (double*)dev_alloc(c, sizeof(double) * (size_t)ld * m);
    c->gm_cs = (double*)dev_alloc(c, sizeof(double) * m);
    c->gm_sn = (double*)dev_alloc(c, sizeof(double) * m);
    c->gm_g = (double*)dev_alloc(c, sizeof(double) * ld);
    c->gm_y = (double*)dev_alloc(c, sizeof(double) * m);
    c->gm_res = (double*)dev_alloc(c, sizeof(double) * 2);
    DD_CUDA(cudaMallocHost(&c->gm_res_h, sizeof(double) * 2));
    c->gm_alloc = m;
  }
  double* W = c->gm_W;
  double* h2 = c->gm_h + ld;        // second Gram-Schmidt pass
  double* nrm2 = c->gm_h + 2 * ld;  // ||w||^2
  const double* const* Vp = c->gm_Vptr;
  auto read_scalar = [&](const double* d) -> double {
    DD_CUDA(cudaMemcpyAsync(c->gm_res_h, d, sizeof(double), cudaMemcpyDeviceToHost, s));
    DD_CUDA(cudaStreamSynchronize(s));
    if (c->timing) timer_collect(c);
    return c->gm_res_h[0];
  };
  PcgState init;
  std::memset(&init, 0, sizeof(init));
  DD_CUDA(cudaMemcpyAsync(c->st, &init, sizeof(init), cudaMemcpyHostToDevice, s));
  // r_0 = b - A x_0
  TIMED(KC_STENCIL, s, launch_stencil(c, c->tabS, c->x, W, s));
  TIMED(KC_XRUPDATE, s, launch_axpby(c, -1.0, W, 1.0, nullptr, b, W, s));
  TIMED(KC_XRUPDATE, s, launch_dot(c, W, W, nrm2, s));
  const double r0 = std::sqrt(read_scalar(nrm2));
  int its = 0;
  double rel = 0.0;
  if (!std::isfinite(r0)) return fail(c, DD_ENAN, "non-finite GMRES residual");
  if (r0 == 0.0) {
    if (iters) *iters = 0;
    if (relres) *relres = 0.0;
    return DD_OK;
  }
  while (true) {
    TIMED(KC_XRUPDATE, s, launch_scale_by_norm(c, W, nrm2, c->gm_V[0], s));
    TIMED(KC_MISC, s, launch_gmres_start(c, nrm2, s));
    int j = 0, done = 0;
    for (j = 0; j < m; ++j) {
      precond(c, c->gm_V[j], 0, c->gm_Z[j]);
      TIMED(KC_STENCIL, s, launch_stencil(c, c->tabS, c->gm_Z[j], W, s));
      TIMED(KC_XRUPDATE, s, launch_multidot(c, j + 1, Vp, W, c->gm_h, 0, s));
      TIMED(KC_XRUPDATE, s, launch_multiaxpy(c, j + 1, Vp, c->gm_h, -1.0, W, s));
      TIMED(KC_XRUPDATE, s, launch_multidot(c, j + 1, Vp, W, h2, 0, s));
      TIMED(KC_XRUPDATE, s, launch_multiaxpy(c, j + 1, Vp, h2, -1.0, W, s));
      TIMED(KC_XRUPDATE, s, launch_add_inplace(c, j + 1, c->gm_h, h2, s));
      TIMED(KC_XRUPDATE, s, launch_dot(c, W, W, nrm2, s));
      TIMED(KC_XRUPDATE, s, launch_scale_by_norm(c, W, nrm2, c->gm_V[j + 1], s));
      TIMED(KC_MISC, s, launch_givens(c, j, s));
      const double est = read_scalar(c->gm_res);
      ++its;
      if (!std::isfinite(est)) return fail(c, DD_ENAN, "non-finite GMRES residual");
      rel = est / r0;
      if (est <= rtol * r0) {
        done = 1;
        ++j;
        break;
      }
      if (its >= maxit) {
        ++j;
        break;
      }
    }
    const int mm = std::min(j, m);
    TIMED(KC_MISC, s, launch_backsolve(c, mm, s));
    TIMED(KC_XRUPDATE, s, launch_multiaxpy(c, mm, c->gm_Zptr, c->gm_y, 1.0, c->x, s));
    // stop on the method's own residual |g_{j+1}| (as PCG stops on its recursive residual);
    // otherwise restart from the true residual
    if (done) break;
    if (its >= maxit) {
      if (iters) *iters = its;
      if (relres) *relres = rel;
      return fail(c, DD_EMAXIT, "GMRES reached maxit");
    }
    TIMED(KC_STENCIL, s, launch_stencil(c, c->tabS, c->x, W, s));
    TIMED(KC_XRUPDATE, s, launch_axpby(c, -1.0, W, 1.0, nullptr, b, W, s));
    TIMED(KC_XRUPDATE, s, launch_dot(c, W, W, nrm2, s));
    if (!std::isfinite(read_scalar(nrm2))) return fail(c, DD_ENAN, "non-finite GMRES residual");
  }
  if (iters) *iters = its;
  if (relres) *relres = rel;
  return DD_OK;
}

// the inner solve of the outer eigen-iterations: PCG (AS2) or GMRES (either preconditioner)
int inner_solve(dd_ctx* c, const double* b, double rtol, int maxit, int* iters, double* relres) {
  if (c->krylov == 1) return gmres_run(c, b, rtol, maxit, iters, relres);
  if (c->ras) throw Error(DD_EINVAL, "the restricted Schwarz preconditioner is not symmetric: use GMRES");
  return pcg_run(c, b, rtol, maxit, iters, relres);
}

void read_outer(dd_ctx* c) {
  DD_CUDA(cudaMemcpyAsync(c->ost_h, c->ost, sizeof(OuterState), cudaMemcpyDeviceToHost, c->stream));
  DD_CUDA(cudaStreamSynchronize(c->stream));
  if (c->timing) timer_collect(c);
}

}  // namespace

// ==========================================================================================
extern "C" {

const char* dd_status_string(int s) {
  switch (s) {
    case DD_OK: return "DD_OK";
    case DD_EINVAL: return "DD_EINVAL";
    case DD_ESTATE: return "DD_ESTATE";
    case DD_ENOMEM: return "DD_ENOMEM";
    case DD_ECUDA: return "DD_ECUDA";
    case DD_ENAN: return "DD_ENAN";
    case DD_ENOTSPD: return "DD_ENOTSPD";
    case DD_EMAXIT: return "DD_EMAXIT";
    case DD_ETIMEOUT: return "DD_ETIMEOUT";
    case DD_EUNSUPPORTED: return "DD_EUNSUPPORTED";
    default: return "DD_UNKNOWN";
  }
}

const char* dd_last_error(const dd_ctx* c) { return c ? c->err.c_str() : g_setup_err.c_str(); }

void dd_destroy(dd_ctx* c) {
  if (!c) return;
  if (c->stream) cudaStreamSynchronize(c->stream);
  if (c->graph) cudaGraphExecDestroy(c->graph);
  dd::gemm_free(c);
  for (void* p : c->allocs) cudaFree(p);
  if (c->st_h) cudaFreeHost(c->st_h);
  if (c->gm_res_h) cudaFreeHost(c->gm_res_h);
  if (c->ost_h) cudaFreeHost(c->ost_h);
  if (c->lst_h) cudaFreeHost(c->lst_h);
  if (c->side) cudaStreamDestroy(c->side);
  if (c->ev_fork) cudaEventDestroy(c->ev_fork);
  if (c->ev_join) cudaEventDestroy(c->ev_join);
  if (c->ev_enter) cudaEventDestroy(c->ev_enter);
  if (c->stream) cudaStreamDestroy(c->stream);
  for (auto& pe : c->timer.pending) {
    cudaEventDestroy(pe.second.first);
    cudaEventDestroy(pe.second.second);
  }
  delete c;
}

int dd_setup(const dd_grid* gr, const double* V, size_t nV, void* stream, dd_ctx** out) {
  if (out) *out = nullptr;
  if (!gr || !V || !out) return fail(nullptr, DD_EINVAL, "null argument");
  const dd_grid G = *gr;
  if (G.p < 1 || G.p > 2) return fail(nullptr, DD_EINVAL, "p must be 1 or 2");
  if (G.q != 1) return fail(nullptr, DD_EINVAL, "q must be 1");
  if (G.L < 1) return fail(nullptr, DD_EINVAL, "L must be >= 1");
  if (G.n < 3) return fail(nullptr, DD_EINVAL, "n must be >= 3");
  const double nyd = G.ell * G.n;
  const int ny = (int)std::lround(nyd);
  if (!(std::fabs(nyd - ny) < 1e-9) || ny < 2) return fail(nullptr, DD_EINVAL, "ell * n must be an integer >= 2");
  if (G.overlap < 1 || 2 * G.overlap >= G.n) return fail(nullptr, DD_EINVAL, "need 1 <= overlap and 2 overlap < n");
  if (G.quad_pts < 1 || G.quad_pts > dd::kMaxQ) return fail(nullptr, DD_EINVAL, "quad_pts must be 1..4");
  if (G.pu_kind != DD_PU_EQUAL && G.pu_kind != DD_PU_DISTANCE) return fail(nullptr, DD_EINVAL, "bad pu_kind");
  if (G.precision < DD_PREC_FP64 || G.precision > DD_PREC_FP8) return fail(nullptr, DD_EINVAL, "bad precision");
  if (G.coarse != 0 && G.coarse != 1) return fail(nullptr, DD_EINVAL, "coarse must be 0 or 1");
  size_t expect = (size_t)ny;
  for (int k = 0; k < G.p; ++k) expect *= (size_t)G.n;
  for (int k = 0; k <= G.p; ++k) expect *= (size_t)G.quad_pts;
  if (nV != expect) return fail(nullptr, DD_EINVAL, "nV does not match n^p ny Q^(p+1)");
  long long cols = 1;
  for (int k = 0; k < G.p; ++k) cols *= (long long)G.L * G.n + 1;
  long long yp = 4;
  while (yp < ny) yp *= 2;
  if (cols * yp > (1LL << 31)) return fail(nullptr, DD_EINVAL, "grid too large");

  dd_ctx* c = nullptr;
  try {
    c = new dd_ctx();
  } catch (...) {
    return fail(nullptr, DD_ENOMEM, "host allocation failed");
  }
  c->grid = G;
  c->user_stream = (cudaStream_t)stream;
  int rc = guarded(c, [&]() -> int {
    DD_CUDA(cudaGetDevice(&c->device));
    DD_CUDA(cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking));
    DD_CUDA(cudaEventCreateWithFlags(&c->ev_enter, cudaEventDisableTiming));
    enter(c);
    Geo& g = c->g;
    g.p = G.p; g.L = G.L; g.n = G.n; g.ny = ny; g.nyi = ny - 1;
    g.delta = G.overlap; g.Q = G.quad_pts;
    g.Ypad = 4;
    g.ylog = 2;
    while (g.Ypad < ny) {
      g.Ypad *= 2;
      g.ylog += 1;
    }
    g.ncx = G.L * G.n + 1;
    g.nxi = G.L * G.n - 1;
    g.ncol = (G.p == 1) ? g.ncx : (long long)g.ncx * g.ncx;
    g.plen = g.ncol * g.Ypad;
    g.ndof = (G.p == 1 ? (long long)g.nxi : (long long)g.nxi * g.nxi) * g.nyi;
    g.nsub = (G.p == 1) ? G.L : G.L * G.L;
    g.ntap = (G.p == 1) ? 9 : 27;
    g.ncls = ((G.p == 1) ? G.n : G.n * G.n) * g.Ypad;
    g.h = 1.0 / G.n;
    DD_CUDA(cudaStreamCreateWithFlags(&c->side, cudaStreamNonBlocking));
    DD_CUDA(cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming));
    DD_CUDA(cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming));
    DD_CUDA(cudaMallocHost(&c->st_h, sizeof(PcgState)));
    DD_CUDA(cudaMallocHost(&c->ost_h, sizeof(OuterState)));
    c->dev_err = (int*)dev_alloc(c, sizeof(int) * 16);
    c->red = (double*)dev_alloc(c, sizeof(double) * kMaxRedBlocks * 4);
    c->cnt = (unsigned*)dev_alloc(c, sizeof(unsigned) * CNT_NUM);
    c->st = (PcgState*)dev_alloc(c, sizeof(PcgState));
    c->ost = (OuterState*)dev_alloc(c, sizeof(OuterState));
    c->Vqp = (double*)dev_alloc(c, sizeof(double) * nV);
    if (is_device_ptr(V)) DD_CUDA(cudaMemcpyAsync(c->Vqp, V, sizeof(double) * nV, cudaMemcpyDeviceToDevice, c->stream));
    else DD_CUDA(cudaMemcpyAsync(c->Vqp, V, sizeof(double) * nV, cudaMemcpyHostToDevice, c->stream));
    launch_check_finite(c->Vqp, (long long)nV, c->dev_err, c->stream);
    int bad = 0;
    DD_CUDA(cudaMemcpyAsync(&bad, c->dev_err, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    DD_CUDA(cudaStreamSynchronize(c->stream));
    if (bad) throw Error(DD_ENAN, "V contains non-finite values");
    const size_t ntab = (size_t)g.ntap * g.ncls;
    c->tabA = (double*)dev_alloc(c, sizeof(double) * ntab);
    c->tabM = (double*)dev_alloc(c, sizeof(double) * ntab);
    c->tabS = (double*)dev_alloc(c, sizeof(double) * ntab);
    c->tabS2 = (float2*)dev_alloc(c, sizeof(float2) * pair_tap_stride(g.p) * g.ncls);
    c->pq_pairs = (pairs_possible(c) && G.precision != DD_PREC_FP64) ? 1 : 0;
    launch_build_tables(c);
    build_subdomains(c);
    c->x = alloc_vec(c);
    c->r = alloc_vec(c);
    c->z = alloc_vec(c);
    c->pb[0] = alloc_vec(c);
    c->pb[1] = alloc_vec(c);
    if (g.p == 2) c->p2 = reinterpret_cast<float2*>(alloc_vec(c));   // 8-byte elements, the vectors' layout
    c->q = alloc_vec(c);
    c->w1 = alloc_vec(c);
    c->w2 = alloc_vec(c);
    c->w3 = alloc_vec(c);
    c->xe = alloc_vec(c);
    c->stage_a = (double*)dev_alloc(c, sizeof(double) * g.ndof);
    c->stage_b = (double*)dev_alloc(c, sizeof(double) * g.ndof);
    c->ncell = (long long)((G.p == 1) ? G.n : G.n * G.n) * g.nyi;
    c->psi_cell = (double*)dev_alloc(c, sizeof(double) * c->ncell);
    c->wT = (double*)dev_alloc(c, sizeof(double) * (size_t)c->ntypes * c->kpad);
    c->puT = (double*)dev_alloc(c, sizeof(double) * (size_t)c->ntypes * c->kpad);
    c->wT32 = (float*)dev_alloc(c, sizeof(float) * (size_t)c->ntypes * c->kpad);
    c->puT32 = (float*)dev_alloc(c, sizeof(float) * (size_t)c->ntypes * c->kpad);
    c->c0 = (double*)dev_alloc(c, sizeof(double) * g.nsub);
    c->u0 = (double*)dev_alloc(c, sizeof(double) * g.nsub);
    c->u0f = (float*)dev_alloc(c, sizeof(float) * g.nsub);
    c->A0band = (double*)dev_alloc(c, sizeof(double) * (size_t)g.nsub * (G.p == 1 ? 3 : 9));
    DD_CUDA(cudaStreamSynchronize(c->stream));
    c->stage = 1;
    return DD_OK;
  });
  if (rc != DD_OK) {
    g_setup_err = c->err;
    dd_destroy(c);
    return rc;
  }
  *out = c;
  return DD_OK;
}

int dd_set_potential(dd_ctx* c, const double* V, size_t nV) {
  if (!V) return fail(c, DD_EINVAL, "null potential");
  int rc = stage_err(c, 1);
  if (rc) return rc;
  size_t expect = (size_t)c->g.ny;
  for (int k = 0; k < c->g.p; ++k) expect *= (size_t)c->g.n;
  for (int k = 0; k <= c->g.p; ++k) expect *= (size_t)c->g.Q;
  if (nV != expect) return fail(c, DD_EINVAL, "nV does not match n^p ny Q^(p+1)");
  return guarded(c, [&]() -> int {
    enter(c);
    if (is_device_ptr(V))
      DD_CUDA(cudaMemcpyAsync(c->Vqp, V, sizeof(double) * nV, cudaMemcpyDeviceToDevice, c->stream));
    else
      DD_CUDA(cudaMemcpyAsync(c->Vqp, V, sizeof(double) * nV, cudaMemcpyHostToDevice, c->stream));
    DD_CUDA(cudaMemsetAsync(c->dev_err, 0, sizeof(int), c->stream));
    launch_check_finite(c->Vqp, (long long)nV, c->dev_err, c->stream);
    int bad = 0;
    DD_CUDA(cudaMemcpyAsync(&bad, c->dev_err, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    DD_CUDA(cudaStreamSynchronize(c->stream));
    if (bad) throw Error(DD_ENAN, "V contains non-finite values");
    launch_build_tables(c);
    DD_CUDA(cudaStreamSynchronize(c->stream));
    reset_graph(c);
    c->stage = 1;
    return DD_OK;
  });
}

long long dd_kernel_launch_count(void) { return dd::launch_count(); }

int dd_cell_eigenpair(dd_ctx* c, double* sigma_out, double* psi_out) {
  int rc = stage_err(c, 1);
  if (rc) return rc;
  return guarded(c, [&]() -> int {
    enter(c);
    int st = cell_eigenpair(c);
    launch_tabS(c, c->sigma);
    launch_coarse_weights(c);
    reset_graph(c);
    if (psi_out) {
      if (is_device_ptr(psi_out))
        DD_CUDA(cudaMemcpyAsync(psi_out, c->psi_cell, sizeof(double) * c->ncell, cudaMemcpyDeviceToDevice, c->stream));
      else
        DD_CUDA(cudaMemcpyAsync(psi_out, c->psi_cell, sizeof(double) * c->ncell, cudaMemcpyDeviceToHost, c->stream));
    }
    DD_CUDA(cudaStreamSynchronize(c->stream));
    if (sigma_out) *sigma_out = c->sigma;
    if (c->stage < 2) c->stage = 2;
    if (st == DD_EMAXIT) return fail(c, DD_EMAXIT, "cell inverse iteration hit its limit");
    return DD_OK;
  });
}

int dd_coarse_build(dd_ctx* c) {
  int rc = stage_err(c, 2);
  if (rc) return rc;
  return guarded(c, [&]() -> int {
    enter(c);
    const Geo& g = c->g;
    reset_graph(c);
    int* flag = c->dev_err + 3;
    DD_CUDA(cudaMemsetAsync(flag, 0, sizeof(int), c->stream));
    const size_t bsz = (size_t)c->ntypes * c->nloc_max * (c->band + 1);
    // the coarse matrix A_0 = Z^T A_sigma Z does not depend on the local factors: it is
    // assembled on the side stream while the local matrices are factored and inverted (those
    // run on a few SMs and leave the GPU mostly idle)
    if (c->grid.coarse) {
      DD_CUDA(cudaEventRecord(c->ev_fork, c->stream));
      DD_CUDA(cudaStreamWaitEvent(c->side, c->ev_fork, 0));
      coarse_assemble(c, c->side);
      DD_CUDA(cudaEventRecord(c->ev_join, c->side));
    }
    if (use_gemm(c)) {
      // the mixed form only forms A_T^{-1} from the factor and rounds it to BF16/TF32/E4M3:
      // an FP32 factor and FP32 solves are far more accurate than that rounding
      if (!c->bandCB32) {
        c->bandCB32 = (float*)dev_alloc(c, sizeof(float) * bsz);
        c->bandRB32 = (float*)dev_alloc(c, sizeof(float) * bsz);
        c->bandInv32 = (float*)dev_alloc(c, sizeof(float) * (size_t)c->ntypes * c->nloc_max);
      }
      launch_local_assemble(c, c->bandCB32);
      launch_band_factor(c, c->bandCB32, c->bandRB32, c->bandInv32, c->ntypes, c->nloc_max, c->band, flag,
                         c->type_nloc);
    } else {
      if (!c->bandCB) {
        c->bandCB = (double*)dev_alloc(c, sizeof(double) * bsz);
        c->bandRB = (double*)dev_alloc(c, sizeof(double) * bsz);
        c->bandInv = (double*)dev_alloc(c, sizeof(double) * (size_t)c->ntypes * c->nloc_max);
      }
      launch_local_assemble(c, c->bandCB);
      launch_band_factor(c, c->bandCB, c->bandRB, c->bandInv, c->ntypes, c->nloc_max, c->band, flag, c->type_nloc);
    }
    int fl = 0;
    DD_CUDA(cudaMemcpyAsync(&fl, flag, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    DD_CUDA(cudaStreamSynchronize(c->stream));
    if (fl) throw Error(DD_ENOTSPD, "local matrix not positive definite");
    if (use_gemm(c)) {
      int r2 = gemm_setup(c);
      if (r2 != DD_OK) return r2;
    } else if (!c->Y64) {
      c->Y64 = (double*)dev_alloc(c, sizeof(double) * (size_t)g.nsub * c->kpad);
    }
    if (c->grid.coarse) {
      DD_CUDA(cudaStreamWaitEvent(c->stream, c->ev_join, 0));
      coarse_factor(c);   // its storage is allocated on the first build and reused
    }
    DD_CUDA(cudaStreamSynchronize(c->stream));
    c->stage = 3;
    return DD_OK;
  });
}

int dd_apply_operator(dd_ctx* c, int op, const double* x, double* y) {
  if (op < 0 || op > 2 || !x || !y) return fail(c, DD_EINVAL, "bad operator or pointer");
  int rc = stage_err(c, op == DD_OP_ASIGMA ? 2 : 1);
  if (rc) return rc;
  return guarded(c, [&]() -> int {
    enter(c);
    const double* tab = op == DD_OP_ASIGMA ? c->tabS : (op == DD_OP_MASS ? c->tabM : c->tabA);
    load_vec(c, x, c->w1);
    launch_stencil(c, tab, c->w1, c->w2, c->stream);
    store_vec(c, c->w2, y);
    DD_CUDA(cudaStreamSynchronize(c->stream));
    return DD_OK;
  });
}

int dd_apply_asigma_pairs(dd_ctx* c, const double* x, double* y) {
  if (!x || !y) return fail(c, DD_EINVAL, "null pointer");
  int rc = stage_err(c, 2);
  if (rc) return rc;
  if (!pairs_possible(c)) return fail(c, DD_EINVAL, "float pairs need at most 256 padded rows for p = 1");
  return guarded(c, [&]() -> int {
    enter(c);
    reset_graph(c);   // the iteration's scalars and vectors are reused here
    // p = z + beta p_{-1} with beta = 0 and p_{-1} = 0: p = x
    PcgState init;
    std::memset(&init, 0, sizeof(init));
    init.rho = 1.0;
    DD_CUDA(cudaMemcpyAsync(c->st, &init, sizeof(init), cudaMemcpyHostToDevice, c->stream));
    DD_CUDA(cudaMemsetAsync(c->pb[0], 0, sizeof(double) * c->g.plen, c->stream));
    load_vec(c, x, c->z);
    const int keep = c->pq_pairs;
    c->pq_pairs = 1;
    try {
      if (c->g.p == 1) {
        launch_fused_pq(c, c->stream);
      } else {
        launch_pupdate_pairs(c, c->stream);
        launch_matvec_pq_pairs(c, c->stream);
      }
    } catch (...) {
      c->pq_pairs = keep;
      throw;
    }
    c->pq_pairs = keep;
    store_vec(c, c->q, y);
    DD_CUDA(cudaStreamSynchronize(c->stream));
    return DD_OK;
  });
}

int dd_apply_preconditioner(dd_ctx* c, const double* r, double* z) {
  if (!r || !z) return fail(c, DD_EINVAL, "null pointer");
  int rc = stage_err(c, 3);
  if (rc) return rc;
  return guarded(c, [&]() -> int {
    enter(c);
    PcgState init;
    std::memset(&init, 0, sizeof(init));
    DD_CUDA(cudaMemcpyAsync(c->st, &init, sizeof(init), cudaMemcpyHostToDevice, c->stream));
    load_vec(c, r, c->r);
    precond(c, c->r, 0);
    store_vec(c, c->z, z);
    DD_CUDA(cudaStreamSynchronize(c->stream));
    if (c->timing) timer_collect(c);
    return DD_OK;
  });
}

int dd_coarse_matrix(dd_ctx* c, double* A0) {
  if (!A0) return fail(c, DD_EINVAL, "null pointer");
  int rc = stage_err(c, 3);
  if (rc) return rc;
  if (!c->grid.coarse) return fail(c, DD_ESTATE, "no coarse space (coarse = 0)");
  return guarded(c, [&]() -> int {
    enter(c);
    const Geo& g = c->g;
    const int N = g.nsub, nnb = (g.p == 1) ? 3 : 9;
    std::vector<double> nb((size_t)N * nnb);
    DD_CUDA(cudaMemcpyAsync(nb.data(), c->A0band, sizeof(double) * nb.size(), cudaMemcpyDeviceToHost, c->stream));
    DD_CUDA(cudaStreamSynchronize(c->stream));
    std::memset(A0, 0, sizeof(double) * (size_t)N * N);
    for (int s = 0; s < N; ++s) {
      const int s1 = (g.p == 1) ? s : s / g.L, s2 = (g.p == 1) ? 0 : s % g.L;
      for (int k = 0; k < nnb; ++k) {
        int t;
        if (g.p == 1) {
          t = s1 + k - 1;
          if (t < 0 || t >= g.L) continue;
        } else {
          const int t1 = s1 + k / 3 - 1, t2 = s2 + k % 3 - 1;
          if (t1 < 0 || t1 >= g.L || t2 < 0 || t2 >= g.L) continue;
          t = t1 * g.L + t2;
        }
        A0[(size_t)s * N + t] = nb[(size_t)s * nnb + k];
      }
    }
    return DD_OK;
  });
}

int dd_pcg_solve(dd_ctx* c, const double* b, double* x, double rtol, int maxit, int* iters_out,
                 double* relres_out) {
  if (!b || !x || !(rtol > 0.0) || maxit < 1) return fail(c, DD_EINVAL, "bad argument");
  int rc = stage_err(c, 3);
  if (rc) return rc;
  return guarded(c, [&]() -> int {
    enter(c);
    if (c->ras) throw Error(DD_EINVAL, "the restricted Schwarz preconditioner is not symmetric: use dd_gmres_solve");
    load_vec(c, b, c->w3);
    load_vec(c, x, c->x);
    int r2 = pcg_run(c, c->w3, rtol, maxit, iters_out, relres_out);
    store_vec(c, c->x, x);
    DD_CUDA(cudaStreamSynchronize(c->stream));
    return r2;
  });
}

int dd_gmres_solve(dd_ctx* c, const double* b, double* x, double rtol, int maxit, int* iters_out,
                   double* relres_out) {
  if (!b || !x || !(rtol > 0.0) || maxit < 1) return fail(c, DD_EINVAL, "bad argument");
  int rc = stage_err(c, 3);
  if (rc) return rc;
  return guarded(c, [&]() -> int {
    enter(c);
    load_vec(c, b, c->w3);
    load_vec(c, x, c->x);
    int r2 = gmres_run(c, c->w3, rtol, maxit, iters_out, relres_out);
    store_vec(c, c->x, x);
    DD_CUDA(cudaStreamSynchronize(c->stream));
    return r2;
  });
}

int dd_inverse_iterate(dd_ctx* c, double* x, double tol_res, double tol_lam, int maxit_outer, double rtol_inner,
                       double* lambda_out, int* outer_out, int* inner_total_out, int* inner_max_out) {
  if (!x || maxit_outer < 1 || !(rtol_inner > 0.0)) return fail(c, DD_EINVAL, "bad argument");
  int rc = stage_err(c, 3);
  if (rc) return rc;
  return guarded(c, [&]() -> int {
    enter(c);
    cudaStream_t s = c->stream;
    const double sigma = c->sigma;
    DD_CUDA(cudaMemsetAsync(c->ost, 0, sizeof(OuterState), s));
    // x_0 -> M-normalised iterate xe, w2 = M xe
    load_vec(c, x, c->w1);
    TIMED(KC_OUTER, s, launch_stencil(c, c->tabM, c->w1, c->w2, s));
    TIMED(KC_OUTER, s, launch_outer_normalize(c, c->w1, c->w2, c->xe, s));
    TIMED(KC_OUTER, s, launch_outer_residual(c, c->xe, c->w2, c->w3, s));
    read_outer(c);
    if (c->ost_h->status != 0) throw Error(c->ost_h->status, "initial vector has zero M-norm");
    double rho_prev = sigma + c->ost_h->xAx;
    double rho = rho_prev;
    int k = 0, inner_tot = 0, inner_max = 0, status = DD_EMAXIT;
    for (k = 1; k <= maxit_outer; ++k) {
      // b = M x_k (in w2); w = A_sigma^{-1} b by PCG from zero
      DD_CUDA(cudaMemsetAsync(c->x, 0, sizeof(double) * c->g.plen, s));
      int it = 0;
      double rel = 0.0;
      int prc = inner_solve(c, c->w2, rtol_inner, 10000, &it, &rel);
      inner_tot += it;
      inner_max = std::max(inner_max, it);
      if (prc != DD_OK && prc != DD_EMAXIT) return prc;
      // x_{k+1} = w / ||w||_M
      TIMED(KC_OUTER, s, launch_stencil(c, c->tabM, c->x, c->w2, s));
      TIMED(KC_OUTER, s, launch_outer_normalize(c, c->x, c->w2, c->xe, s));
      TIMED(KC_OUTER, s, launch_outer_residual(c, c->xe, c->w2, c->w3, s));
      read_outer(c);
      if (c->ost_h->status != 0) throw Error(c->ost_h->status, "outer normalisation failed");
      rho = sigma + c->ost_h->xAx;
      const double eta = std::sqrt(c->ost_h->rr / c->ost_h->mm) / std::fabs(rho);
      if (!std::isfinite(rho)) throw Error(DD_ENAN, "non-finite Rayleigh quotient");
      if (eta <= tol_res && std::fabs(rho - rho_prev) <= tol_lam * std::fabs(rho)) {
        status = DD_OK;
        break;
      }
      rho_prev = rho;
    }
    store_vec(c, c->xe, x);
    DD_CUDA(cudaStreamSynchronize(s));
    if (lambda_out) *lambda_out = rho;
    if (outer_out) *outer_out = std::min(k, maxit_outer);
    if (inner_total_out) *inner_total_out = inner_tot;
    if (inner_max_out) *inner_max_out = inner_max;
    if (status != DD_OK) return fail(c, status, "outer iteration limit reached");
    return DD_OK;
  });
}

int dd_lopcg(dd_ctx* c, double* x, int inner, double tol_res, double tol_lam, int maxit_outer, double rtol_inner,
             double* lambda_out, int* outer_out, int* inner_total_out, int* inner_max_out) {
  if (!x || maxit_outer < 1) return fail(c, DD_EINVAL, "bad argument");
  if (inner != DD_INNER_FIXED && inner != DD_INNER_ADAPTIVE && inner != DD_INNER_FUSED)
    return fail(c, DD_EINVAL, "inner must be DD_INNER_FIXED, DD_INNER_ADAPTIVE or DD_INNER_FUSED");
  if (inner == DD_INNER_FIXED && !(rtol_inner > 0.0)) return fail(c, DD_EINVAL, "rtol_inner must be > 0");
  int rc = stage_err(c, 3);
  if (rc) return rc;
  return guarded(c, [&]() -> int {
    enter(c);
    cudaStream_t s = c->stream;
    const Geo& g = c->g;
    const double sigma = c->sigma;
    if (!c->lst) {
      c->lst = (LopState*)dev_alloc(c, sizeof(LopState));
      DD_CUDA(cudaMallocHost(&c->lst_h, sizeof(LopState)));
      c->lop_red = (double*)dev_alloc(c, sizeof(double) * kMaxRedBlocks * 15);
      for (double*& v : c->lop) v = alloc_vec(c);
    }
    // work vectors: iterate, previous iterate, spare; their A_sigma- and M-images (and two
    // spares for the next images); the images of w; the outer residual
    double *X = c->lop[0], *XP = c->lop[1], *T = c->lop[2];
    double *AX = c->lop[3], *AXP = c->lop[4], *MX = c->lop[5], *MXP = c->lop[6];
    double *AW = c->lop[7], *MW = c->lop[8], *RO = c->lop[9], *AT = c->lop[10], *MT = c->lop[11];
    for (double* v : c->lop) DD_CUDA(cudaMemsetAsync(v, 0, sizeof(double) * g.plen, s));
    DD_CUDA(cudaMemsetAsync(c->ost, 0, sizeof(OuterState), s));
    DD_CUDA(cudaMemsetAsync(c->lst, 0, sizeof(LopState), s));
    // x_0 = e_1 (first interior node), B-normalised, and its images
    const long long first = (g.p == 1) ? (long long)g.Ypad : ((long long)g.ncx + 1) * g.Ypad;
    launch_set_entry(XP, first, 1.0, s);
    TIMED(KC_OUTER, s, launch_stencil(c, c->tabM, XP, MXP, s));
    TIMED(KC_OUTER, s, launch_lop_normalize(c, XP, MXP, s));
    TIMED(KC_OUTER, s, launch_stencil(c, c->tabS, XP, AXP, s));
    // x_1 from the caller, B-normalised; A_sigma x_1, rho and the outer residual (explicit)
    auto explicit_images = [&]() {
      TIMED(KC_OUTER, s, launch_stencil(c, c->tabM, X, MX, s));
      TIMED(KC_OUTER, s, launch_lop_normalize(c, X, MX, s));
      TIMED(KC_OUTER, s, launch_outer_residual(c, X, MX, AX, s, RO));
      read_outer(c);
      if (c->ost_h->status != 0) throw Error(c->ost_h->status, "iterate has zero M-norm");
    };
    load_vec(c, x, X);
    explicit_images();
    double lam = c->ost_h->xAx, rr = c->ost_h->rr, mm = c->ost_h->mm;
    bool exact = true;   // images computed by stencils (not carried as combinations)
    double rho_prev = std::numeric_limits<double>::infinity(), rho = sigma + lam;
    int k = 0, inner_tot = 0, inner_max = 0, status = DD_EMAXIT;
    for (k = 0; k <= maxit_outer; ++k) {
      rho = sigma + lam;
      if (!std::isfinite(rho)) throw Error(DD_ENAN, "non-finite Rayleigh quotient");
      const double eta = std::sqrt(rr / mm) / std::fabs(rho);
      if (eta <= tol_res && std::fabs(rho - rho_prev) <= tol_lam * std::fabs(rho)) {
        if (exact) {
          status = DD_OK;
          break;
        }
        // confirm on images recomputed from x (the carried ones hold rounding of k steps)
        explicit_images();
        exact = true;
        lam = c->ost_h->xAx;
        rr = c->ost_h->rr;
        mm = c->ost_h->mm;
        const double rho_e = sigma + lam;
        const double eta_e = std::sqrt(rr / mm) / std::fabs(rho_e);
        if (eta_e <= tol_res && std::fabs(rho_e - rho_prev) <= tol_lam * std::fabs(rho_e)) {
          rho = rho_e;
          status = DD_OK;
          break;
        }
      }
      if (k == maxit_outer) break;
      // inner step: A_sigma w = r_o inexactly (Algorithm 1), or w = M^{-1} r_o (fused)
      const double* W = nullptr;
      int it = 0;
      if (inner == DD_INNER_FUSED) {
        PcgState init;
        std::memset(&init, 0, sizeof(init));
        DD_CUDA(cudaMemcpyAsync(c->st, &init, sizeof(init), cudaMemcpyHostToDevice, s));
        precond(c, RO, 0);
        W = c->z;
        it = 1;
      } else {
        const double rt = (inner == DD_INNER_FIXED) ? rtol_inner : std::min(0.1, std::sqrt(rr));
        DD_CUDA(cudaMemsetAsync(c->x, 0, sizeof(double) * g.plen, s));
        double rel = 0.0;
        const int prc = inner_solve(c, RO, rt, 10000, &it, &rel);
        if (prc != DD_OK && prc != DD_EMAXIT) return prc;
        W = c->x;
      }
      inner_tot += it;
      inner_max = std::max(inner_max, it);
      TIMED(KC_OUTER, s, launch_stencil2(c, c->tabS, c->tabM, W, AW, MW, s));
      // Rayleigh-Ritz on span{x_k, w_k, x_{k-1}}; x_{k+1} = S c with its images and r_o
      const double* S[3] = {X, W, XP};
      const double* AS[3] = {AX, AW, AXP};
      const double* MS[3] = {MX, MW, MXP};
      TIMED(KC_RR, s, launch_lop_gram(c, S, AS, MS, 1e-10, s));
      TIMED(KC_RR, s, launch_lop_update3(c, S, AS, MS, T, AT, MT, RO, s));
      // rotate: x_{k-1} <- x_k, x_k <- x_{k+1}, and the same for the images
      double* t0 = XP;
      XP = X;
      X = T;
      T = t0;
      t0 = AXP;
      AXP = AX;
      AX = AT;
      AT = t0;
      t0 = MXP;
      MXP = MX;
      MX = MT;
      MT = t0;
      DD_CUDA(cudaMemcpyAsync(c->lst_h, c->lst, sizeof(LopState), cudaMemcpyDeviceToHost, s));
      DD_CUDA(cudaStreamSynchronize(s));
      if (c->timing) timer_collect(c);
      if (c->lst_h->status != 0) throw Error(c->lst_h->status, "Rayleigh-Ritz step failed");
      rho_prev = rho;
      lam = c->lst_h->theta;
      rr = c->lst_h->rr;
      mm = c->lst_h->mm;
      exact = false;
    }
    // keep the buffer roles for the next call
    c->lop[0] = X; c->lop[1] = XP; c->lop[2] = T;
    c->lop[3] = AX; c->lop[4] = AXP; c->lop[5] = MX; c->lop[6] = MXP;
    c->lop[10] = AT; c->lop[11] = MT;
    store_vec(c, X, x);
    DD_CUDA(cudaStreamSynchronize(s));
    if (lambda_out) *lambda_out = rho;
    if (outer_out) *outer_out = std::min(k, maxit_outer);
    if (inner_total_out) *inner_total_out = inner_tot;
    if (inner_max_out) *inner_max_out = inner_max;
    if (status != DD_OK) return fail(c, status, "outer iteration limit reached");
    return DD_OK;
  });
}

namespace {

// Projected PCG for the adjoint (A - lambda M) w = r, r orthogonal to phi, w M-orthogonal to
// phi: the preconditioned residual is projected, z = Pi M^{-1} Pi^T r with
// Pi = I - phi (M phi)^T, so every search direction stays in the M-orthogonal complement
// of phi, where A - lambda M is positive definite even when lambda and phi carry the error
// of the eigen-solve (there A - lambda M has a tiny negative eigenvalue along phi).
// Polak-Ribiere beta (exact for the FP64 preconditioner, flexible for the rounded one).
// Vectors: b (in, overwritten as the residual), x (out), u = M phi, phi; scratch p, q, rp.
int adjoint_pcg(dd_ctx* c, double* r, double* x, const double* u, const double* phi, double* p, double* q,
                double* zs, double rtol, int maxit, int* iters) {
  cudaStream_t s = c->stream;
  const Geo& g = c->g;
  double* d = c->gscal;   // device scalars
  auto dot = [&](const double* a, const double* b2) -> double {
    launch_dot(c, a, b2, d, s);
    double h = 0.0;
    DD_CUDA(cudaMemcpyAsync(&h, d, sizeof(double), cudaMemcpyDeviceToHost, s));
    DD_CUDA(cudaStreamSynchronize(s));
    return h;
  };
  auto axpby = [&](double a, const double* xv, double bcoef, const double* yv, double* out) {
    launch_axpby(c, a, xv, bcoef, nullptr, yv, out, s);
  };
  auto apply_prec = [&]() {   // zs = Pi M^{-1} Pi^T r  (r is kept orthogonal to phi)
    PcgState init;
    std::memset(&init, 0, sizeof(init));
    DD_CUDA(cudaMemcpyAsync(c->st, &init, sizeof(init), cudaMemcpyHostToDevice, s));
    precond(c, r, 0);
    const double t = dot(u, c->z);
    axpby(1.0, c->z, -t, phi, zs);
  };
  DD_CUDA(cudaMemsetAsync(x, 0, sizeof(double) * g.plen, s));
  const double rr0 = dot(r, r);
  *iters = 0;
  if (rr0 == 0.0) return DD_OK;
  apply_prec();
  DD_CUDA(cudaMemcpyAsync(p, zs, sizeof(double) * g.plen, cudaMemcpyDeviceToDevice, s));
  double rz = dot(r, zs);
  for (int k = 1; k <= maxit; ++k) {
    TIMED(KC_STENCIL, s, launch_stencil(c, c->tabL, p, q, s));
    const double pq = dot(p, q);
    if (!(pq > 0.0)) return fail(c, std::isfinite(pq) ? DD_ENOTSPD : DD_ENAN, "adjoint: p^T (A - lambda M) p <= 0");
    const double alpha = rz / pq;
    axpby(1.0, x, alpha, p, x);
    axpby(1.0, r, -alpha, q, r);
    // keep r orthogonal to phi against drift
    const double tp = dot(phi, r);
    axpby(1.0, r, -tp, u, r);
    const double rr = dot(r, r);
    *iters = k;
    if (rr <= rtol * rtol * rr0) return DD_OK;
    apply_prec();
    const double zq = dot(zs, q);
    const double rz_new = dot(r, zs);
    const double beta = -zq / pq;   // (z_{k+1}, r_{k+1} - r_k) / (z_k, r_k)
    axpby(1.0, zs, beta, p, p);
    rz = rz_new;
  }
  return fail(c, DD_EMAXIT, "adjoint PCG reached maxit");
}

}  // namespace

int dd_potential_gradient(dd_ctx* c, const double* phi, double lambda, double g_lambda, const double* g_phi,
                          double rtol, double* dV, size_t nV, int* iters_out) {
  if (!phi || !dV || !(rtol > 0.0)) return fail(c, DD_EINVAL, "bad argument");
  int rc = stage_err(c, 3);
  if (rc) return rc;
  const Geo& g = c->g;
  size_t expect = (size_t)(g.p == 2 ? g.n * g.n : g.n) * (size_t)(g.nyi + 1);
  for (int k = 0; k < g.p + 1; ++k) expect *= (size_t)g.Q;
  if (nV != expect) return fail(c, DD_EINVAL, "nV does not match n^p ny Q^(p+1)");
  return guarded(c, [&]() -> int {
    enter(c);
    cudaStream_t s = c->stream;
    if (!c->gv[0]) {
      for (double*& v : c->gv) v = alloc_vec(c);
      c->tabL = (double*)dev_alloc(c, sizeof(double) * (size_t)g.ncls * g.ntap);
      c->gscal = (double*)dev_alloc(c, sizeof(double) * 2);
      c->gout = (double*)dev_alloc(c, sizeof(double) * nV);
    }
    double *PHI = c->gv[0], *G = c->gv[1], *U = c->gv[2], *VV = c->gv[3];
    double *W = c->gv[4], *P = c->gv[5], *Q = c->gv[6], *Z = c->gv[7];
    load_vec(c, phi, PHI);
    int iters = 0;
    if (g_phi) {
      // r = g - M phi (phi^T g): orthogonal to phi, the right-hand side of the adjoint
      load_vec(c, g_phi, G);
      TIMED(KC_OUTER, s, launch_stencil(c, c->tabM, PHI, U, s));
      TIMED(KC_OUTER, s, launch_dot(c, PHI, G, c->gscal, s));
      TIMED(KC_OUTER, s, launch_axpby(c, 1.0, G, -1.0, c->gscal, U, G, s));
      launch_tab_shift(c, lambda, c->tabL);
      const int prc = adjoint_pcg(c, G, W, U, PHI, P, Q, Z, rtol, 10000, &iters);
      if (prc != DD_OK) return prc;
      // w <- w - phi (M phi)^T w (the iterates stay there up to rounding)
      TIMED(KC_OUTER, s, launch_dot(c, U, W, c->gscal, s));
      TIMED(KC_OUTER, s, launch_axpby(c, 1.0, W, -1.0, c->gscal, PHI, W, s));
      // v = g_lambda phi - w
      TIMED(KC_OUTER, s, launch_axpby(c, g_lambda, PHI, -1.0, nullptr, W, VV, s));
    } else {
      TIMED(KC_OUTER, s, launch_axpby(c, g_lambda, PHI, 0.0, nullptr, PHI, VV, s));
    }
    // dV[e, q] = sum over copies of h^d W_q phi_h (g_lambda phi_h - w_h)
    double* out = is_device_ptr(dV) ? dV : c->gout;
    TIMED(KC_OUTER, s, launch_qp_product(c, PHI, VV, out, s));
    if (out != dV) DD_CUDA(cudaMemcpyAsync(dV, out, sizeof(double) * nV, cudaMemcpyDeviceToHost, s));
    DD_CUDA(cudaStreamSynchronize(s));
    if (iters_out) *iters_out = iters;
    return DD_OK;
  });
}

int dd_eigenpair(const dd_grid* g, const double* V, size_t nV, void* stream, double* lambda_out, double* phi_out,
                 double* sigma_out) {
  dd_ctx* c = nullptr;
  int rc = dd_setup(g, V, nV, stream, &c);
  if (rc) return rc;
  rc = dd_cell_eigenpair(c, sigma_out, nullptr);
  if (rc == DD_OK) rc = dd_coarse_build(c);
  if (rc == DD_OK) {
    rc = guarded(c, [&]() -> int {
      // x_0 = 1 in the context's staging buffer (device), phi written to phi_out
      launch_fill(c->stage_b, c->g.ndof, 1.0, c->stream);
      DD_CUDA(cudaStreamSynchronize(c->stream));
      return DD_OK;
    });
  }
  if (rc == DD_OK) {
    double* xv = c->stage_b;
    rc = dd_inverse_iterate(c, xv, 1e-8, 1e-10, 100, 1e-8, lambda_out, nullptr, nullptr, nullptr);
    if ((rc == DD_OK || rc == DD_EMAXIT) && phi_out) {
      int rc2 = guarded(c, [&]() -> int {
        if (is_device_ptr(phi_out))
          DD_CUDA(cudaMemcpyAsync(phi_out, xv, sizeof(double) * c->g.ndof, cudaMemcpyDeviceToDevice, c->stream));
        else
          DD_CUDA(cudaMemcpyAsync(phi_out, xv, sizeof(double) * c->g.ndof, cudaMemcpyDeviceToHost, c->stream));
        DD_CUDA(cudaStreamSynchronize(c->stream));
        return DD_OK;
      });
      if (rc == DD_OK) rc = rc2;
    }
  }
  if (rc != DD_OK) g_setup_err = c->err;
  dd_destroy(c);
  return rc;
}

int dd_query(const dd_ctx* c, dd_info* info) {
  if (!c || !info) return DD_EINVAL;
  info->ndof = c->g.ndof;
  info->ncell = c->ncell;
  info->nsub = c->g.nsub;
  info->ntypes = c->ntypes;
  info->nloc_max = c->nloc_max;
  info->kpad = c->kpad;
  info->band_local = c->band;
  info->sigma = c->sigma;
  info->cell_iters = c->cell_iters;
  info->stage = c->stage;
  info->device_bytes = c->bytes;
  info->gemm_tile_n = c->gemm_ok ? (c->gemm_bn_opt != 0 ? c->gemm_bn_opt : c->gemm_bn) : 0;
  info->reserved_ = 0;
  return DD_OK;
}

int dd_set_option(dd_ctx* c, int option, int value) {
  if (!c) return DD_EINVAL;
  switch (option) {
    case DD_OPT_CHECK_EVERY:
      if (value < 1 || value > 1000) return fail(c, DD_EINVAL, "check_every out of range");
      c->check_every = value;
      break;
    case DD_OPT_USE_GRAPH: c->use_graph = value ? 1 : 0; break;
    case DD_OPT_FLEXIBLE:
      if (value < -1 || value > 1) return fail(c, DD_EINVAL, "flexible must be -1, 0 or 1");
      c->flexible_opt = value;
      break;
    case DD_OPT_TIMING: c->timing = value ? 1 : 0; break;
    case DD_OPT_KRYLOV:
      if (value != 0 && value != 1) return fail(c, DD_EINVAL, "krylov must be 0 (PCG) or 1 (GMRES)");
      c->krylov = value;
      break;
    case DD_OPT_PRECOND:
      if (value != 0 && value != 1) return fail(c, DD_EINVAL, "precond must be 0 (AS2) or 1 (RAS2)");
      c->ras = value;
      break;
    case DD_OPT_RESTART:
      if (value < 1 || value > 200) return fail(c, DD_EINVAL, "restart must be in 1..200");
      if (c->gm_alloc != 0 && c->gm_alloc != value) return fail(c, DD_ESTATE, "restart fixed after the first GMRES solve");
      c->gm_restart = value;
      break;
    case DD_OPT_COARSE_SOLVE:
      if (value < 0 || value > 2) return fail(c, DD_EINVAL, "coarse solve must be 0, 1 or 2");
      if (value == 1 && c->g.p == 2) return fail(c, DD_EINVAL, "cyclic reduction needs p = 1");
      c->coarse_mode = value;
      break;
    case DD_OPT_FUSED_PQ:
      if (value < -1 || value > 2) return fail(c, DD_EINVAL, "fused p update must be -1, 0, 1 or 2");
      if (value >= 1 && c->g.p == 2) return fail(c, DD_EINVAL, "the fused p update and stencil needs p = 1");
      c->fused_pq_opt = value;
      if (!fuse_xr_possible(c)) c->fuse_xr = 0;
      break;
    case DD_OPT_FUSE_XR:
      if (value < -1 || value > 1) return fail(c, DD_EINVAL, "fused x/r update must be -1, 0 or 1");
      if (value == 1 && !fuse_xr_possible(c))
        return fail(c, DD_EINVAL, "the fused x/r update needs p = 1, BF16 or TF32 local inverses, the fused p "
                                  "update and at most 4096 subdomains");
      c->fuse_xr_opt = value;
      c->fuse_xr = value > 0 ? 1 : 0;
      break;
    case DD_OPT_TILED3:
      if (value != 0 && value != 1) return fail(c, DD_EINVAL, "tiled p = 2 matvec must be 0 or 1");
      c->matvec_tiled = value;
      break;
    case DD_OPT_X_LAG:
      if (value != 0 && value != 1) return fail(c, DD_EINVAL, "deferred x update must be 0 or 1");
      c->x_lag = value;
      break;
    case DD_OPT_PDL:
      if (value != 0 && value != 1) return fail(c, DD_EINVAL, "programmatic dependent launch must be 0 or 1");
      c->pdl = value;
      break;
    case DD_OPT_PAIRS:
      if (value < -1 || value > 1) return fail(c, DD_EINVAL, "float pairs must be -1, 0 or 1");
      if (value == 1 && !pairs_possible(c))
        return fail(c, DD_EINVAL, "float pairs need at most 256 padded rows for p = 1");
      c->pq_pairs_opt = value;
      c->pq_pairs = value >= 0 ? value : ((pairs_possible(c) && c->grid.precision != DD_PREC_FP64) ? 1 : 0);
      break;
    case DD_OPT_PROLONG_TABLES:
      if (value != 0 && value != 1) return fail(c, DD_EINVAL, "prolong tables must be 0 or 1");
      c->prolong_tables_opt = value;
      c->prolong_arith = (c->prolong_closed && !value) ? 1 : 0;
      break;
    case DD_OPT_GEMM_TILE_N:
      if (value != 0 && value != 128 && value != 160 && value != 256)
        return fail(c, DD_EINVAL, "GEMM tile N must be 0, 128, 160 or 256");
      c->gemm_bn_opt = value;
      break;
    case DD_OPT_LOCAL_RHS: {
      if (value != 0 && value != 1 && value != 2 && value != 4)
        return fail(c, DD_EINVAL, "local right-hand sides per warp must be 0, 1, 2 or 4");
      const int kmax = rhs_per_warp(c->nloc_max, c->band);
      const int k = value == 0 ? std::min(2, kmax) : std::min(value, kmax);
      try {
        set_local_groups(c, k);
      } catch (const Error& e) {
        return fail(c, e.code, e.msg);
      }
      break;
    }
    default: return fail(c, DD_EINVAL, "unknown option");
  }
  reset_graph(c);
  return DD_OK;
}

int dd_kernel_timings(dd_ctx* c, int* count, const char** names, long long* launches, double* ms) {
  if (!c || !count) return DD_EINVAL;
  *count = dd::KC_COUNT;
  for (int k = 0; k < dd::KC_COUNT; ++k) {
    if (names) names[k] = dd::kClassNames[k];
    if (launches) launches[k] = c->timer.launches[k];
    if (ms) ms[k] = c->timer.ms[k];
  }
  return DD_OK;
}

int dd_reset_timings(dd_ctx* c) {
  if (!c) return DD_EINVAL;
  for (int k = 0; k < dd::KC_COUNT; ++k) {
    c->timer.launches[k] = 0;
    c->timer.ms[k] = 0.0;
  }
  return DD_OK;
}

}  // extern "C"
