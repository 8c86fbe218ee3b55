// Batched ground states: many independent instances (uneven L, own potential and shift), each
// with its own context and private stream, driven by a pool of host threads so that their
// kernels run concurrently on the GPU.  Instances are taken largest first (longest
// processing time first keeps the tail short); each worker runs the whole pipeline of its
// instance (cell eigenpair, coarse build, outer iteration) and records its wall time.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <mutex>
#include <thread>
#include <vector>

#include "dd_internal.h"

struct dd_batch {
  std::vector<dd_ctx*> ctx;
  std::vector<double*> x;      // per instance: device start vector / solution (ndof)
  std::vector<long long> ndof;
  int device = 0;
};

namespace {

__global__ void k_fill(long long n, double v, double* x) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n;
       t += (long long)gridDim.x * blockDim.x)
    x[t] = v;
}

void destroy_all(dd_batch* b) {
  for (double* p : b->x)
    if (p) cudaFree(p);
  for (dd_ctx* c : b->ctx) dd_destroy(c);
  delete b;
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
  *out = b;
  return DD_OK;
}

int dd_batch_size(const dd_batch* b) { return b ? (int)b->ctx.size() : 0; }

dd_ctx* dd_batch_context(dd_batch* b, int i) {
  if (!b || i < 0 || i >= (int)b->ctx.size()) return nullptr;
  return b->ctx[i];
}

int dd_batch_ground_states(dd_batch* b, int method, int threads, double* lambda_out, double* const* phi_out,
                           int* outer_out, int* inner_out, double* seconds_out) {
  if (!b) return DD_EINVAL;
  if (method < DD_BATCH_IPM || method > DD_BATCH_LOPCG_ADAPTIVE) return DD_EINVAL;
  const int n = (int)b->ctx.size();
  if (threads < 1) threads = std::min(n, 16);
  threads = std::min(threads, n);
  std::vector<int> order(n);
  for (int i = 0; i < n; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](int a, int c) { return b->ndof[a] > b->ndof[c]; });
  std::atomic<int> next{0};
  std::atomic<int> first_error{DD_OK};
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
      const auto t0 = std::chrono::steady_clock::now();
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
      if (rc == DD_OK) {
        if (method == DD_BATCH_IPM)
          rc = dd_inverse_iterate(c, b->x[i], 1e-8, 1e-10, 100, 1e-8, &lam, &outer, &tot, &mx);
        else
          rc = dd_lopcg(c, b->x[i], method == DD_BATCH_LOPCG_FUSED ? DD_INNER_FUSED : DD_INNER_ADAPTIVE, 1e-8,
                        1e-10, 1000, 1e-8, &lam, &outer, &tot, &mx);
      }
      if (rc == DD_OK && phi_out && phi_out[i]) {
        if (cudaMemcpyAsync(phi_out[i], b->x[i], sizeof(double) * (size_t)b->ndof[i], cudaMemcpyDefault, s) !=
                cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess) {
          cudaGetLastError();
          rc = DD_ECUDA;
        }
      }
      const double sec = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
      if (lambda_out) lambda_out[i] = lam;
      if (outer_out) outer_out[i] = outer;
      if (inner_out) inner_out[i] = tot;
      if (seconds_out) seconds_out[i] = sec;
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
  return first_error.load();
}

void dd_batch_destroy(dd_batch* b) {
  if (b) destroy_all(b);
}

}  // extern "C"
