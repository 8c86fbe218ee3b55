// Throughput self-test of the FP64 and FP32 fused multiply-add pipes.
//
// The FP64 vector kernels of the iteration (the stencil, the x/r update, the dot products)
// issue more FP64 FMAs per byte than GB300's narrow FP64 pipe retires at HBM speed, so their
// roofline is that pipe's rate, and the mixed form's FP32 node values are bounded by the FP32
// pipe.  This kernel measures both on the GPU at hand: every thread runs kChains independent
// chains a <- a * b + c (no dependence between chains, so the pipe, not the FMA latency, bounds
// it), over a grid of 8 blocks of 256 threads per SM; the result is 2 flops per FMA over the
// CUDA-event time of the launch.
#include <cuda_runtime.h>

#include <algorithm>

#include "dd_internal.h"

namespace dd {

constexpr int kChains = 8;

// b and c are moved into registers per thread: a uniform (constant-bank) operand form of the
// FMA measured 16% below the pipe's rate on GB300 (1.058 against 1.257 TFLOP/s in FP64)
template <typename T>
__global__ void __launch_bounds__(256) k_fma_peak(int iters, T b0, T c0, T* out) {
  const T b = b0 + (T)1e-12 * (T)(threadIdx.x & 7), c = c0 * ((T)1 + (T)1e-9 * (T)(threadIdx.x & 3));
  T a[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) a[k] = (T)(threadIdx.x + k);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = fma(a[k], b, c);
  }
  T s = 0;
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += a[k];
  out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = s;   // keeps every chain live
}

}  // namespace dd

extern "C" int dd_alu_peak_test(int kind, int reps, double* tflops_out) {
  using namespace dd;
  if ((kind != 0 && kind != 1) || reps < 1 || reps > 100 || !tflops_out) return DD_EINVAL;
  *tflops_out = 0.0;
  void* out = nullptr;
  cudaStream_t s = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int rc = DD_OK;
  try {
    int dev = 0, sms = 0;
    DD_CUDA(cudaGetDevice(&dev));
    DD_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int threads = 256, blocks = sms * 8;
    const int iters = kind == 0 ? 4096 : 131072;   // about 10-20 ms per launch on GB300
    DD_CUDA(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
    DD_CUDA(cudaEventCreate(&e0));
    DD_CUDA(cudaEventCreate(&e1));
    DD_CUDA(cudaMalloc(&out, (size_t)blocks * threads * 8));
    double best = 0.0;
    for (int r = 0; r <= reps; ++r) {   // the first launch is an untimed warm-up
      DD_CUDA(cudaEventRecord(e0, s));
      if (kind == 0)
        (k_fma_peak<double><<<blocks, threads, 0, s>>>(iters, 0.999999, 1e-7, (double*)out), note_launch());
      else
        (k_fma_peak<float><<<blocks, threads, 0, s>>>(iters, 0.999999f, 1e-7f, (float*)out), note_launch());
      DD_CUDA(cudaGetLastError());
      DD_CUDA(cudaEventRecord(e1, s));
      DD_CUDA(cudaEventSynchronize(e1));
      float ms = 0.f;
      DD_CUDA(cudaEventElapsedTime(&ms, e0, e1));
      const double flops = 2.0 * kChains * (double)iters * threads * blocks;
      if (r > 0 && ms > 0.f) best = std::max(best, flops / (ms * 1e-3) / 1e12);
    }
    *tflops_out = best;
  } catch (const Error& e) {
    rc = e.code;
  }
  if (out) cudaFree(out);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (s) cudaStreamDestroy(s);
  return rc;
}
