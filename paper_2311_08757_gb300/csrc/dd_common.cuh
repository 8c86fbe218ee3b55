// Device helpers shared by the kernels: reductions, index maps, stencil evaluation.
#pragma once

#include <cuda_bf16.h>

#include "dd_internal.h"

namespace dd {

constexpr int kThreads = 256;
constexpr unsigned kFull = 0xffffffffu;

// Last-block counters (one per reduction site so that concurrent kernels never share one).
enum CounterId {
  CNT_PQ = 0, CNT_RR, CNT_RZ, CNT_INIT, CNT_DOT0, CNT_DOT1, CNT_OUTER0, CNT_OUTER1, CNT_OUTER2, CNT_LOP, CNT_GRAD, CNT_CELL,
  CNT_NUM = 16
};
constexpr int kMaxRedBlocks = 4096;   // partial slots per value

// Tree sum over the warp (result in lane 0).  GB300 issues FP64 at 2 lanes per clock per
// SM and charges a whole warp instruction whatever its active mask (measured: predicated
// adds execute on all 32 lanes), so every step costs a full warp's FP64 issue.
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(kFull, v, o);
  return v;
}

// Sums NV values over the block; the result is valid in thread 0 only.  For up to four
// values and blocks of at most 256 threads (a multiple of 32), the partials are staged in
// shared memory and one warp adds them: (warps - 1) + 5 FP64 warp instructions per value
// instead of 5 per warp plus 5 (12 against 45 for 256 threads).
template <int NV>
__device__ __forceinline__ void block_sum(double (&v)[NV]) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  if constexpr (NV <= 4) {
    if (blockDim.x <= 256 && (blockDim.x & 31) == 0) {
      __shared__ double st[NV][256];
#pragma unroll
      for (int k = 0; k < NV; ++k) st[k][threadIdx.x] = v[k];
      __syncthreads();
      if (wid == 0) {
#pragma unroll
        for (int k = 0; k < NV; ++k) {
          double a = st[k][lane];
          for (int w = 1; w < nw; ++w) a += st[k][lane + 32 * w];
          v[k] = warp_sum(a);
        }
      }
      __syncthreads();
      return;
    }
  }
  __shared__ double sm[32][NV];
#pragma unroll
  for (int k = 0; k < NV; ++k) v[k] = warp_sum(v[k]);
  __syncthreads();
  if (lane == 0)
#pragma unroll
    for (int k = 0; k < NV; ++k) sm[wid][k] = v[k];
  __syncthreads();
  if (wid == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      double t = lane < nw ? sm[lane][k] : 0.0;
      v[k] = warp_sum(t);
    }
  }
  __syncthreads();
}

// Programmatic dependent launch (launch_chain with pdl set): pdl_wait blocks until the
// preceding kernel on the stream has completed and its writes are visible; pdl_trigger lets
// the following kernel's blocks be scheduled (it takes effect once every block of this grid has
// issued it or exited).  Both do nothing in a plain launch.  The chain's kernels issue both
// first thing, before reading anything a predecessor wrote.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
__device__ __forceinline__ void pdl_enter() {
  pdl_wait();
  pdl_trigger();
}

// PCG direction double buffer: iteration k (k = completed iterations) reads p_{k-1} from
// pb[k & 1] and writes p_k to pb[(k + 1) & 1].
__device__ __forceinline__ const double* p_prev(const double* pb0, const double* pb1, int k) {
  return (k & 1) ? pb1 : pb0;
}
__device__ __forceinline__ double* p_cur(double* pb0, double* pb1, int k) { return (k & 1) ? pb0 : pb1; }

// A block's place in the launch of one problem: block b of nb.  A plain launch is one
// problem (b = blockIdx.x, nb = gridDim.x); a batched launch runs the blocks of several
// problems' launches side by side, each block with the index and count it would have had
// in its own problem's launch, so every problem's arithmetic (and the order of its
// reductions) is that of its plain launch.
struct VBlk {
  int b, nb;
};
__device__ __forceinline__ VBlk vblk_self() { return VBlk{(int)blockIdx.x, (int)gridDim.x}; }

// Deterministic grid-wide sum: every block stores its partial; the last block to finish
// adds the partials in block order and returns true (result in tot[] of thread 0).
template <int NV>
__device__ __forceinline__ bool grid_sum_last(double (&v)[NV], double* partials, unsigned* counter,
                                              double (&tot)[NV], VBlk vb) {
  __shared__ int s_last;
  block_sum<NV>(v);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) partials[(size_t)k * kMaxRedBlocks + vb.b] = v[k];
    __threadfence();
    unsigned t = atomicAdd(counter, 1u);
    s_last = (t == (unsigned)vb.nb - 1);
  }
  __syncthreads();
  if (!s_last) return false;
  __threadfence();
  double s[NV];
#pragma unroll
  for (int k = 0; k < NV; ++k) {
    s[k] = 0.0;
    for (int b = threadIdx.x; b < vb.nb; b += blockDim.x)
      s[k] += __ldcg(partials + (size_t)k * kMaxRedBlocks + b);
  }
  block_sum<NV>(s);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) tot[k] = s[k];
    *counter = 0u;
  }
  return true;
}
template <int NV>
__device__ __forceinline__ bool grid_sum_last(double (&v)[NV], double* partials, unsigned* counter,
                                              double (&tot)[NV]) {
  return grid_sum_last<NV>(v, partials, counter, tot, vblk_self());
}

// ---- precision conversions on the integer pipe ------------------------------------------
// GB300 retires FP64 instructions (conversions included) at 2 per clock per SM; these
// conversions do the same rounding with integer operations for normal-range values.

// Out-of-line fallbacks for non-normal values (kept out of line so that they are not
// if-converted into the common path).
static __device__ __noinline__ unsigned short bf16_bits_slow(double x) {
  const __nv_bfloat16 h = __double2bfloat16(x);
  return *reinterpret_cast<const unsigned short*>(&h);
}
static __device__ __noinline__ float tf32_slow(double x) {
  unsigned r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"((float)x));
  return __uint_as_float(r);
}
static __device__ __noinline__ double f64_slow(float f) { return (double)f; }

// IEEE round-to-nearest-even of a double to bfloat16 (bits).  Only 32-bit integer
// operations on the two words of x; results outside the normal range, infinities and NaNs
// take the hardware conversion (one range check selects them).  Zeros, which every padded
// column holds, are answered inside that branch by their sign bit, without the call.
__device__ __forceinline__ unsigned short f64_to_bf16_bits(double x) {
  const unsigned hi = (unsigned)__double2hiint(x), lo = (unsigned)__double2loint(x);
  const int eb = (int)((hi >> 20) & 0x7FFu) - 1023 + 127;
  if (__builtin_expect((unsigned)(eb - 1) >= 254u, 0)) {
    if (((hi << 1) | lo) == 0u) return (unsigned short)(hi >> 16);   // +-0
    return bf16_bits_slow(x);
  }
  const unsigned keep = (hi >> 13) & 0x7Fu;   // top 7 of the 52 mantissa bits
  const unsigned remh = hi & 0x1FFFu;         // the other 45 bits are remh:lo; half is 0x1000:0
  unsigned r = ((unsigned)eb << 7) | keep;
  const bool above = remh > 0x1000u || (remh == 0x1000u && lo != 0u);
  const bool tie = remh == 0x1000u && lo == 0u;
  if (above || (tie && (keep & 1u))) r += 1;   // a carry rounds into the exponent
  return (unsigned short)(((hi >> 31) << 15) | r);
}

// Round-to-nearest, ties away from zero, of a double to TF32 (an FP32 bit pattern whose low
// 13 mantissa bits are zero), as cvt.rna.tf32.f32 would round the exact value.  Integer
// operations as above (zeros too).
__device__ __forceinline__ float f64_to_tf32(double x) {
  const unsigned hi = (unsigned)__double2hiint(x);
  const int ef = (int)((hi >> 20) & 0x7FFu) - 1023 + 127;
  if (__builtin_expect((unsigned)(ef - 1) >= 254u, 0)) {
    if (((hi << 1) | (unsigned)__double2loint(x)) == 0u) return __uint_as_float(hi & 0x80000000u);   // +-0
    return tf32_slow(x);
  }
  const unsigned keep = (hi >> 10) & 0x3FFu;   // top 10 mantissa bits
  unsigned r = ((unsigned)ef << 10) | keep;
  if ((hi & 0x3FFu) >= 0x200u) r += 1;         // the other 42 bits at or above half
  return __uint_as_float(((hi >> 31) << 31) | (r << 13));
}

// Exact float -> double by integer operations for normal floats and zeros; subnormals,
// infinities and NaNs take the hardware conversion.
__device__ __forceinline__ double f32_to_f64(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned e = (u >> 23) & 0xFFu;
  if (__builtin_expect(e - 1u >= 254u, 0)) {
    if ((u << 1) == 0u) return __hiloint2double((int)(u & 0x80000000u), 0);   // +-0
    return f64_slow(f);
  }
  const unsigned m = u & 0x7FFFFFu;
  const unsigned hi = (u & 0x80000000u) | ((e + 896u) << 20) | (m >> 3);
  return __hiloint2double((int)hi, (int)(m << 29));
}

// ---- float pairs: FP64 values carried as hi + lo on the FP32 pipe ---------------------
// A pair (hi, lo) of floats stands for hi + lo (48 significand bits).  Products of pairs are
// formed with the FMA error-free product (Dekker's two-product: a*b = p + fma(a, b, -p)
// exactly), sums of the leading parts with Knuth's two-sum (s = a + b exactly as s + err);
// the error terms and the cross products hi*lo' + lo*hi' are carried in the low word.  The
// explicit _rn intrinsics keep the compiler from contracting the error-free steps.

static __device__ __noinline__ float2 f64_split_slow(double d) {
  const float hi = __double2float_rz(d);
  return make_float2(hi, __double2float_rz(d - (double)hi));
}

// d = hi + lo + e with |e| < 2^-47 |d|: hi is d's first 24 significand bits, lo the next 24
// (both truncated toward zero).  Integer operations on the two words of d for
// 2^-74 <= |d| < 2^127 (so that lo stays a normal float) and zeros; other values (tiny,
// huge, subnormal, infinities, NaNs) take the hardware conversions.
__device__ __forceinline__ float2 f64_split(double d) {
  const unsigned H = (unsigned)__double2hiint(d), Lw = (unsigned)__double2loint(d);
  const unsigned E = (H >> 20) & 0x7FFu;
  if (__builtin_expect(E - 949u > 1150u - 949u, 0)) {
    if (((H << 1) | Lw) == 0u) return make_float2(0.0f, 0.0f);
    return f64_split_slow(d);
  }
  const unsigned sgn = H & 0x80000000u;
  // exponent rebias 1023 -> 127 (896 << 20) and the 20 + 3 leading significand bits
  const float hi = __uint_as_float(sgn | ((H - 0x38000000u) << 3) | (Lw >> 29));
  // the remaining 29 bits: normalise to bit 31, keep 24 (the leading one lands on the
  // exponent field's lowest bit, hence E - 918 - lz rather than E - 917 - lz)
  const unsigned m29 = Lw & 0x1FFFFFFFu;
  const unsigned lz = __clz((int)m29);
  const unsigned lo_bits = sgn | (((E - 918u - lz) << 23) + ((m29 << lz) >> 8));
  return make_float2(hi, __uint_as_float(m29 ? lo_bits : 0u));
}

// (s, c) += (th + tl) * (xh + xl): s the running leading sum, c the low-order accumulator
__device__ __forceinline__ void pair_fma(float th, float tl, float xh, float xl, float& s, float& c) {
  const float p = __fmul_rn(th, xh);
  const float e = __fmaf_rn(th, xh, -p);                   // th * xh = p + e exactly
  const float u = __fadd_rn(s, p);
  const float bv = __fsub_rn(u, s);
  const float err = __fadd_rn(__fsub_rn(s, __fsub_rn(u, bv)), __fsub_rn(p, bv));   // s + p = u + err
  s = u;
  c = __fadd_rn(c, __fadd_rn(e, err));
  c = __fmaf_rn(th, xl, c);
  c = __fmaf_rn(tl, xh, c);
}

// Subdomain-local vectors stored in the kpad-strided arrays (rounded local inverses,
// restrictions, local results, coarse and partition-of-unity weights) keep the column
// padding of the global vectors: local column cc, slot sj sits at cc * Ypad + sj, so a
// subdomain's restriction is a contiguous run of the padded global vector (p = 1) or w1 such
// runs (p = 2).  The banded factors and the FP64 solves use the compact order cc * nyi + sj.
__device__ __forceinline__ int loc_pad(const Geo& g, int k) { return (k / g.nyi) * g.Ypad + k % g.nyi; }

// Interior-element enumeration of a padded vector: t in [0, nxi^p * Ypad).
struct Node {
  long long idx;   // padded index
  int slot;        // y slot (j - 1); >= nyi means pad
  int a1, a2;      // node columns (a2 = 0 for p = 1)
};

template <int P>
__device__ __forceinline__ Node node_of(const Geo& g, long long t) {
  Node nd;
  long long u = t >> g.ylog;
  nd.slot = (int)(t & (g.Ypad - 1));
  if (P == 1) {
    nd.a1 = 1 + (int)u;
    nd.a2 = 0;
    nd.idx = t + g.Ypad;
  } else {
    int q1 = (int)(u / g.nxi);
    nd.a1 = 1 + q1;
    nd.a2 = 1 + (int)(u - (long long)q1 * g.nxi);
    nd.idx = ((long long)nd.a1 * g.ncx + nd.a2) * g.Ypad + nd.slot;
  }
  return nd;
}

template <int P>
__device__ __forceinline__ int cls_of(const Geo& g, const Node& nd) {
  if (P == 1) return (nd.a1 % g.n) * g.Ypad + nd.slot;
  return ((nd.a1 % g.n) * g.n + (nd.a2 % g.n)) * g.Ypad + nd.slot;
}

// y(node) = sum over the 3^d taps of tab[tap][cls] x(node + offset(tap)).
template <int P>
__device__ __forceinline__ double stencil_at(const Geo& g, const double* __restrict__ tab,
                                             const double* __restrict__ x, long long idx, int cls) {
  double acc = 0.0;
  if (P == 1) {
    const long long cs = g.Ypad;
#pragma unroll
    for (int dx = -1; dx <= 1; ++dx)
#pragma unroll
      for (int dy = -1; dy <= 1; ++dy) {
        const int tap = (dx + 1) * 3 + (dy + 1);
        acc = fma(__ldg(tab + (size_t)tap * g.ncls + cls), x[idx + dx * cs + dy], acc);
      }
  } else {
    const long long c1 = (long long)g.ncx * g.Ypad, c2 = g.Ypad;
#pragma unroll
    for (int d1 = -1; d1 <= 1; ++d1)
#pragma unroll
      for (int d2 = -1; d2 <= 1; ++d2)
#pragma unroll
        for (int dy = -1; dy <= 1; ++dy) {
          const int tap = ((d1 + 1) * 3 + (d2 + 1)) * 3 + (dy + 1);
          acc = fma(__ldg(tab + (size_t)tap * g.ncls + cls), x[idx + d1 * c1 + d2 * c2 + dy], acc);
        }
  }
  return acc;
}

// Owners of an interior node column along one axis: subdomains i with lo(i) <= a <= hi(i).
__device__ __forceinline__ int axis_owners(const Geo& g, int a, int (&own)[2], int (&loc)[2]) {
  int k = 0;
  int i0 = a / g.n - 1;
  for (int i = i0; i <= i0 + 2; ++i) {
    if (i < 0 || i >= g.L) continue;
    int lo = ax_lo(g, i), hi = ax_hi(g, i);
    if (a >= lo && a <= hi && k < 2) {
      own[k] = i;
      loc[k] = a - lo;
      ++k;
    }
  }
  return k;
}

}  // namespace dd
