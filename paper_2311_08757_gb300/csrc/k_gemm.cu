// Local solves as a batched dense contraction on the tensor cores (tcgen05, sm_103a).
//
// Two-level additive Schwarz (Sec. 3.1) needs y_i = A_{sigma,i}^{-1} R_i r for every
// subdomain.  Subdomains of one type share A_T = A_{sigma,i}, so with the rows
// R_i r stacked (type-sorted) into B_T (N_T x K) the local solves of a type are one GEMM
//     Y_T[n][m] = sum_k Ainv_T[m][k] B_T[n][k]           (Ainv_T symmetric, K-major)
// with Ainv_T rounded to BF16 or TF32 and FP32 accumulation.  The rounding makes the
// preconditioner inexact; the outer Krylov method is then flexible CG.
//
// Kernel: one CTA per 128 x BN output tile; warp 0 lane 0 issues TMA loads into a ring of
// 128B-swizzled shared-memory stages (one or two 128-byte swizzle atoms of K each), warp 1
// lane 0 issues tcgen05.mma with the accumulator in tensor memory, all four warps read it
// back with tcgen05.ld and store Y (FP32).  Every mbarrier wait is bounded; on expiry the CTA records an error in a
// device word, stops issuing work and returns after freeing its tensor memory.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp8.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <new>
#include <mutex>
#include <string>

#include <atomic>

#include "dd_async.cuh"
#include "dd_band.cuh"

namespace dd {

struct Tile {
  int type, m0, n0, nend;
};

template <typename T, int BN_ = 256>
struct TcCfg {
  static constexpr int BM = 128, BN = BN_;
  static constexpr int BK = 128 / (int)sizeof(T);   // K of one 128-byte swizzle atom
  static constexpr int UK = 32 / (int)sizeof(T);    // K of one tcgen05.mma (32 bytes)
  // Swizzle atoms per stage and stages.  A stage costs a fixed round trip (full barrier,
  // MMA issue, commit, empty barrier, TMA issue) of about 600 cycles whatever its size, more
  // than the tensor time of one atom (about 460 cycles for 128 x 160 x 64), so the 128 x 160
  // tile moves two atoms per stage in 3 stages (217 KB): its K loop at L = 2048, h = 1/32
  // went from 6.3 to 5.0 us, the tensor floor of the tile shape.  128 x 256 tiles: one atom,
  // 4 stages (193 KB); 128 x 128 tiles: one atom, 3 stages (97 KB), so that two CTAs share
  // an SM and one's epilogue overlaps the other's MMAs.
  static constexpr int ATOMS = (BN_ == 160) ? 2 : 1;
  static constexpr int STAGES = (BN_ == 128 || BN_ == 160) ? 3 : 4;
  // TMEM is allocated in powers of two of at least 32 columns (one FP32 column per output column)
  static constexpr int TMEM_COLS = BN_ <= 32 ? 32 : (BN_ <= 64 ? 64 : (BN_ <= 128 ? 128 : 256));
  static constexpr int A_ATOM = BM * 128;
  static constexpr int B_ATOM = BN * 128;
  static constexpr int A_BYTES = A_ATOM * ATOMS;
  static constexpr int B_BYTES = B_ATOM * ATOMS;
  static constexpr int STAGE_BYTES = A_BYTES + B_BYTES;
  static constexpr int SMEM = STAGES * STAGE_BYTES + 1024 + 256;
};

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* tm, int c0, int c1, uint32_t mbar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
          dst),
      "l"(tm), "r"(c0), "r"(c1), "r"(mbar)
      : "memory");
}

// shared-memory matrix descriptor: K-major operand, 128-byte swizzle, 8-row groups 1024 B apart
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)1 << 16;              // leading byte offset (unused with 128B swizzle, K-major)
  d |= (uint64_t)(1024 >> 4) << 32;    // stride byte offset
  d |= (uint64_t)1 << 46;              // descriptor version
  d |= (uint64_t)2 << 61;              // 128-byte swizzle
  return d;
}

// instruction descriptor: D = F32, A/B format fmt (1 = BF16, 2 = TF32, 0 = E4M3), K-major both, M = 128, N = BN
__host__ __device__ constexpr uint32_t mma_idesc(uint32_t fmt, int M, int N) {
  return (1u << 4) | (fmt << 7) | (fmt << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

template <typename T>
__device__ __forceinline__ void mma_issue(uint32_t tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc);

template <>
__device__ __forceinline__ void mma_issue<__nv_bfloat16>(uint32_t tmem, uint64_t a, uint64_t b, uint32_t idesc,
                                                         uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(
          tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

template <>
__device__ __forceinline__ void mma_issue<float>(uint32_t tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(
          tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

template <>
__device__ __forceinline__ void mma_issue<__nv_fp8_e4m3>(uint32_t tmem, uint64_t a, uint64_t b, uint32_t idesc,
                                                         uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n}\n" ::"r"(
          tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

// operand format field of the instruction descriptor: BF16 1 (kind::f16), TF32 2 (kind::tf32),
// E4M3 0 (kind::f8f6f4)
template <typename T>
constexpr uint32_t mma_fmt() {
  return sizeof(T) == 2 ? 1u : (sizeof(T) == 4 ? 2u : 0u);
}

__device__ __forceinline__ void mma_commit(uint32_t mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar) : "memory");
}

// 16 consecutive FP32 columns of this warp's 32 TMEM lanes; complete after tmem_ld_wait
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t* r) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
}
__device__ __forceinline__ void tmem_ld_wait() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

constexpr int ERR_TMA_WAIT = 1 << 4, ERR_MMA_WAIT = 1 << 5, ERR_ACC_WAIT = 1 << 6;

// The CTA's tile (16-byte aligned), loaded by a volatile instruction so that it is issued
// before the converged-flag test rather than after it: the two L2 round trips overlap.
__device__ __forceinline__ Tile load_tile(const Tile* p) {
  Tile t;
  asm volatile("ld.global.nc.v4.s32 {%0, %1, %2, %3}, [%4];"
               : "=r"(t.type), "=r"(t.m0), "=r"(t.n0), "=r"(t.nend)
               : "l"(p));
  return t;
}

template <typename T, int BN>
__global__ void __launch_bounds__(128, 1)
    k_tc_gemm(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
              const Tile* __restrict__ tiles, int K, int mlimit, int rows_per_type, float* __restrict__ Y,
              int ldy, int* err, const PcgState* st, const float* __restrict__ ysc,
              const PcgState* const* __restrict__ tile_st) {
  using C = TcCfg<T, BN>;
  constexpr int kTmemCols = C::TMEM_COLS;
  pdl_enter();
  const Tile tl = load_tile(tiles + blockIdx.x);
  // a grouped launch over several problems' tiles gives each tile its problem's state
  if (tile_st != nullptr) st = tile_st[blockIdx.x];
  if (st != nullptr && st->done) return;
  extern __shared__ uint8_t smem_raw[];
  const uint32_t raw = smem_u32(smem_raw);
  const uint32_t base = (raw + 1023u) & ~1023u;
  uint8_t* sm = smem_raw + (base - raw);
  const uint32_t sA0 = base;
  const uint32_t sB0 = base + C::STAGES * C::A_BYTES;
  uint8_t* bar_ptr = sm + C::STAGES * C::STAGE_BYTES;
  const uint32_t bar = base + C::STAGES * C::STAGE_BYTES;
  // barriers: full[s] at bar + 8 s, empty[s] at bar + 64 + 8 s, accum at bar + 128, tmem slot at bar + 192
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bar_ptr + 192);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  if (threadIdx.x == 0) {
    for (int s = 0; s < C::STAGES; ++s) {
      mbar_init(bar + 8 * s, 1);
      mbar_init(bar + 64 + 8 * s, 1);
    }
    mbar_init(bar + 128, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;
  const int natoms = K / C::BK;
  const int nk = (natoms + C::ATOMS - 1) / C::ATOMS;   // stages; the last may hold fewer atoms
  const int rowA = tl.type * rows_per_type + tl.m0;

  if (warp == 0 && lane == 0) {
    // producer
    for (int kb = 0; kb < nk; ++kb) {
      const int s = kb % C::STAGES;
      const uint32_t ph = (uint32_t)(kb / C::STAGES) & 1u;
      const int na = min(C::ATOMS, natoms - kb * C::ATOMS);
      if (!mbar_wait(bar + 64 + 8 * s, ph ^ 1u, err, ERR_TMA_WAIT)) break;
      mbar_expect_tx(bar + 8 * s, (uint32_t)(na * (C::A_ATOM + C::B_ATOM)));
      for (int a = 0; a < na; ++a) {
        const int k0 = (kb * C::ATOMS + a) * C::BK;
        tma_load_2d(sA0 + s * C::A_BYTES + a * C::A_ATOM, &tmA, k0, rowA, bar + 8 * s);
        tma_load_2d(sB0 + s * C::B_BYTES + a * C::B_ATOM, &tmB, k0, tl.n0, bar + 8 * s);
      }
    }
  } else if (warp == 1 && lane == 0) {
    // MMA issuer
    constexpr uint32_t fmt = mma_fmt<T>();
    constexpr uint32_t idesc = mma_idesc(fmt, C::BM, C::BN);
    bool ok = true;
    for (int kb = 0; kb < nk && ok; ++kb) {
      const int s = kb % C::STAGES;
      const uint32_t ph = (uint32_t)(kb / C::STAGES) & 1u;
      if (!mbar_wait(bar + 8 * s, ph, err, ERR_MMA_WAIT)) {
        ok = false;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const int na = min(C::ATOMS, natoms - kb * C::ATOMS);
      for (int a = 0; a < na; ++a) {
#pragma unroll
        for (int kk = 0; kk < C::BK / C::UK; ++kk) {
          const uint64_t ad = sw128_desc(sA0 + s * C::A_BYTES + a * C::A_ATOM + kk * 32);
          const uint64_t bd = sw128_desc(sB0 + s * C::B_BYTES + a * C::B_ATOM + kk * 32);
          mma_issue<T>(tmem, ad, bd, idesc, (kb | a | kk) != 0 ? 1u : 0u);
        }
      }
      mma_commit(bar + 64 + 8 * s);
    }
    mma_commit(bar + 128);
  }
  __syncwarp();
  // epilogue: warp w owns TMEM lanes 32w..32w+31 (output rows m)
  const bool ready = mbar_wait(bar + 128, 0, err, ERR_ACC_WAIT);
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (ready) {
    // 32 columns per wait (two loads in flight): 1.9 -> 1.6 us for the 128 x 160 tile
    const int m = tl.m0 + warp * 32 + lane;
    const uint32_t trow = tmem + ((uint32_t)(warp * 32) << 16);
    for (int c0 = 0; c0 < C::BN; c0 += 32) {
      if (tl.n0 + c0 >= tl.nend) break;
      uint32_t r[32];
      tmem_ld16(trow + (uint32_t)c0, r);
      if (c0 + 16 < C::BN) tmem_ld16(trow + (uint32_t)(c0 + 16), r + 16);
      tmem_ld_wait();
      if (m < mlimit) {
#pragma unroll
        for (int j = 0; j < 32; ++j) {
          const int n = tl.n0 + c0 + j;
          // scaled operands (FP8): undo the row scales of A and B
          if (c0 + j < C::BN && n < tl.nend)
            Y[(size_t)n * ldy + m] = ysc != nullptr ? __uint_as_float(r[j]) * ysc[n] : __uint_as_float(r[j]);
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
  }
}

// ----------------------------------------------------------------------------------------
// Host side: tensor maps through the driver entry point (no link-time libcuda dependency).
// ----------------------------------------------------------------------------------------
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_fn() {
  // resolved once (thread-safe initialisation of a function-local static)
  static const EncodeTiledFn fn = []() -> EncodeTiledFn {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !p) {
      cudaGetLastError();
      return nullptr;
    }
    return (EncodeTiledFn)p;
  }();
  if (!fn) throw Error(DD_ECUDA, "cuTensorMapEncodeTiled unavailable");
  return fn;
}

static void make_tmap(CUtensorMap* tm, void* base, int es, int inner, long long rows, int box_inner, int box_rows) {
  cuuint64_t dims[2] = {(cuuint64_t)inner, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)inner * es};
  cuuint32_t box[2] = {(cuuint32_t)box_inner, (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  const CUtensorMapDataType dt = es == 1 ? CU_TENSOR_MAP_DATA_TYPE_UINT8
                                : (es == 2 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32);
  CUresult r = encode_fn()(tm, dt, 2, base,
                           dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                           CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) throw Error(DD_ECUDA, "cuTensorMapEncodeTiled failed (" + std::to_string((int)r) + ")");
}

template <typename T, int BN = 256>
static void launch_tc(const CUtensorMap* tA, const CUtensorMap* tB, const Tile* tiles, int ntiles, int K,
                      int mlimit, int rows_per_type, float* Y, int ldy, int* err, const PcgState* st,
                      cudaStream_t s, const float* ysc = nullptr, const PcgState* const* tile_st = nullptr,
                      bool pdl = false) {
  static PerDeviceOnce attr;   // once per device and instance
  once_per_device(attr, [] {
    DD_CUDA(cudaFuncSetAttribute(k_tc_gemm<T, BN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 TcCfg<T, BN>::SMEM));
  });
  launch_chain(k_tc_gemm<T, BN>, dim3(ntiles), dim3(128), TcCfg<T, BN>::SMEM, s, pdl, *tA, *tB, tiles, K, mlimit,
               rows_per_type, Y, ldy, err, st, ysc, tile_st);
}

// ----------------------------------------------------------------------------------------
// Rounded local inverses from the banded factors: column col of A_T^{-1} (identity
// right-hand side) = row col (symmetric), rounded to BF16 or TF32.
// ----------------------------------------------------------------------------------------
// rounding of FP64 values to the operand type, on the integer pipe (see dd_common.cuh)
template <typename T>
__device__ __forceinline__ T round_fast(double v);
template <>
__device__ __forceinline__ __nv_bfloat16 round_fast<__nv_bfloat16>(double v) {
  const unsigned short b = f64_to_bf16_bits(v);
  return *reinterpret_cast<const __nv_bfloat16*>(&b);
}
template <>
__device__ __forceinline__ float round_fast<float>(double v) {
  return f64_to_tf32(v);
}
template <>
__device__ __forceinline__ double round_fast<double>(double v) {
  return v;
}

// E4M3 (saturating, nearest even) of a scaled value
__device__ __forceinline__ __nv_fp8_e4m3 to_e4m3(double v) {
  __nv_fp8_e4m3 q;
  q.__x = __nv_cvt_double_to_fp8(v, __NV_SATFINITE, __NV_E4M3);
  return q;
}
constexpr double kE4M3Max = 448.0;   // largest finite E4M3 value

// rounding of an FP32 solve result to the operand type (FP64: exact widening, for the FP8
// path's scaling pass)
template <typename T>
__device__ __forceinline__ T round_f32(float v);
template <>
__device__ __forceinline__ __nv_bfloat16 round_f32<__nv_bfloat16>(float v) { return __float2bfloat16_rn(v); }
template <>
__device__ __forceinline__ float round_f32<float>(float v) {
  unsigned r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(v));
  return __uint_as_float(r);
}
template <>
__device__ __forceinline__ double round_f32<double>(float v) { return f32_to_f64(v); }

// Columns of A_T^{-1} by band solves of identity columns with the FP32 factor (the mixed
// form: the result is rounded to the GEMM's operand type right away), one warp per column.
template <typename T, int NV, int PF, int K>
__global__ void k_local_inverse(const int* __restrict__ nloc, int nmax, int b, const float* __restrict__ CB,
                                const float* __restrict__ RB, const float* __restrict__ inv, int ntypes, int kpad,
                                int nyi, int ylog, T* __restrict__ out) {
  extern __shared__ float xs_all[];
  const int wpb = blockDim.x >> 5, wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int groups_per_type = (nmax + K - 1) / K;
  const long long job = (long long)blockIdx.x * wpb + wid;
  if (job >= (long long)ntypes * groups_per_type) return;
  const int ty = (int)(job / groups_per_type);
  const int col0 = (int)(job % groups_per_type) * K;
  const int n = nloc[ty];
  if (col0 >= n) return;
  constexpr int RING = band_ring_elems<NV, PF>();
  float* xs = xs_all + (size_t)wid * (K * nmax + RING);
  float* ring = xs + (size_t)K * nmax;
#pragma unroll
  for (int j = 0; j < K; ++j)
    for (int k = lane; k < n; k += 32) xs[(size_t)j * nmax + k] = (k == col0 + j) ? 1.0f : 0.0f;
  const size_t off = (size_t)ty * nmax;
  band_solve_k<NV, PF, K>(xs, nmax, n, b, CB + off * (b + 1), RB + off * (b + 1), inv + off, ring);
  __syncwarp();
  // rows and columns at their column-padded local positions (the pad rows and columns stay 0)
  auto lp = [&](int k) { return ((k / nyi) << ylog) + k % nyi; };
  for (int j = 0; j < K && col0 + j < n; ++j) {
    T* row = out + ((size_t)ty * kpad + lp(col0 + j)) * kpad;
    for (int k = lane; k < n; k += 32) row[lp(k)] = round_f32<T>(xs[(size_t)j * nmax + k]);
  }
}

// R_i r rounded, subdomain rows in type-sorted order, zero tail up to kpad; the coarse
// right-hand side c_i = (D_i R_i psi)^T r (Def. 2.1) is formed in FP64 in the same pass.
// In the column-padded local layout a subdomain is w1 contiguous runs of w2 * Ypad values of
// r (one run for p = 1), so the block streams them two values per thread and step (pad slots
// of r are zero, and so are the weights there).  Block per subdomain.
// FP8: the row is scaled by s_i = 448 / max|R_i r| before rounding, and 1 / (s_i s_T) (with
// s_T the scale of the type's inverse) is recorded for the GEMM's epilogue.
template <typename T>
__device__ __forceinline__ void store2(T* row, int k, double a, double b, double scale);
template <>
__device__ __forceinline__ void store2<__nv_bfloat16>(__nv_bfloat16* row, int k, double a, double b, double) {
  const unsigned w = (unsigned)f64_to_bf16_bits(a) | ((unsigned)f64_to_bf16_bits(b) << 16);
  *reinterpret_cast<unsigned*>(row + k) = w;
}
template <>
__device__ __forceinline__ void store2<float>(float* row, int k, double a, double b, double) {
  *reinterpret_cast<float2*>(row + k) = make_float2(f64_to_tf32(a), f64_to_tf32(b));
}
template <>
__device__ __forceinline__ void store2<__nv_fp8_e4m3>(__nv_fp8_e4m3* row, int k, double a, double b, double scale) {
  row[k] = to_e4m3(a * scale);
  row[k + 1] = to_e4m3(b * scale);
}

template <typename T>
__device__ __forceinline__ void pack_body(Geo g, const Sub* __restrict__ subs, const int* __restrict__ slot_of,
                                          const double* __restrict__ r, int kpad, T* __restrict__ out,
                                          const double* __restrict__ wT, double* c0, const PcgState* st,
                                          const float* __restrict__ ascale, float* __restrict__ ysc, int s) {
  if (st != nullptr && st->done) return;
  constexpr bool FP8 = sizeof(T) == 1;
  const Sub sb = subs[s];
  const int slot = slot_of[s];
  T* row = out + (size_t)slot * kpad;
  const double* wt = wT + (size_t)sb.type * kpad;
  const int run = sb.w2 * g.Ypad, npair = sb.w1 * run / 2;   // run length is even (Ypad >= 4)
  auto src = [&](int kp) -> long long {   // padded global index of local kp
    const int c1 = kp / run, j = kp - c1 * run;
    return (g.p == 1) ? (long long)(sb.lo1 + c1) * g.Ypad + j
                      : ((long long)(sb.lo1 + c1) * g.ncx + sb.lo2) * g.Ypad + j;
  };
  double scale = 1.0;
  if (FP8) {
    double mx[1] = {0.0};
    for (int e = threadIdx.x; e < npair; e += blockDim.x) {
      const double2 v = *reinterpret_cast<const double2*>(r + src(2 * e));
      mx[0] = fmax(mx[0], fmax(fabs(v.x), fabs(v.y)));
    }
    __shared__ double s_mx[32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int o = 16; o > 0; o >>= 1) mx[0] = fmax(mx[0], __shfl_xor_sync(kFull, mx[0], o));
    if (lane == 0) s_mx[warp] = mx[0];
    __syncthreads();
    double m = 0.0;
    for (int w = 0; w < nw; ++w) m = fmax(m, s_mx[w]);
    scale = m > 0.0 ? kE4M3Max / m : 1.0;
    if (threadIdx.x == 0) ysc[slot] = (float)(ascale[sb.type] / scale);
  }
  double acc[1] = {0.0};
  for (int e = threadIdx.x; e < npair; e += blockDim.x) {
    const int kp = 2 * e;
    const double2 v = *reinterpret_cast<const double2*>(r + src(kp));
    const double2 w = *reinterpret_cast<const double2*>(wt + kp);
    acc[0] = fma(w.x, v.x, acc[0]);
    acc[0] = fma(w.y, v.y, acc[0]);
    store2<T>(row, kp, v.x, v.y, scale);
  }
  for (int kp = 2 * npair + 2 * threadIdx.x; kp < kpad; kp += 2 * blockDim.x) store2<T>(row, kp, 0.0, 0.0, 1.0);
  if (c0 != nullptr) {
    block_sum<1>(acc);
    if (threadIdx.x == 0) c0[s] = acc[0];
  }
}

// A p = 1 PCG iteration's x, r update fused into the restriction packing (BF16/TF32
// operands).  Block s forms r_new = r - alpha q over its subdomain's run of the padded vector
// (the FMA of the separate x/r update), rounds r_new into its packed row and the coarse
// right-hand side, and on the node columns it owns -- a with min(a / n, L - 1) = s, so each
// column once -- updates x += alpha p and adds r_new^2 to (r, r) (FP64).  r itself is written by the prolong-sum that follows (each node once, the same
// FMA), because the neighbouring blocks still read the old r of the columns they share.  The
// last block to finish takes the stop test.
template <typename T>
__device__ __forceinline__ void pack_xr_body(VBlk vb, Geo g, const Sub* __restrict__ subs,
                                             const int* __restrict__ slot_of, const double* __restrict__ r,
                                             const double* __restrict__ q, double* __restrict__ x, double* pb0,
                                             double* pb1, int kpad, T* __restrict__ out,
                                             const double* __restrict__ wT, double* c0, PcgState* st,
                                             double* partials, unsigned* counter) {
  if (st->done) return;
  const int s = vb.b;
  const double alpha = st->alpha;
  const double* __restrict__ p = p_cur(pb0, pb1, st->iter);
  const Sub sb = subs[s];
  T* row = out + (size_t)slot_of[s] * kpad;
  const double* wt = wT + (size_t)sb.type * kpad;
  const int Y = g.Ypad;
  const int npair = sb.w1 * Y / 2;   // p = 1: the restriction is one run of w1 columns
  const long long g0 = (long long)sb.lo1 * Y;
  const int own_lo = max(1, s * g.n), own_hi = (s == g.L - 1) ? g.nxi : (s + 1) * g.n - 1;
  const int e_lo = (own_lo - sb.lo1) * Y / 2, e_hi = (own_hi + 1 - sb.lo1) * Y / 2;
  double rr[1] = {0.0}, acc[1] = {0.0};
  for (int e = threadIdx.x; e < npair; e += blockDim.x) {
    const int kp = 2 * e;
    const long long gi = g0 + kp;
    double2 rv = *reinterpret_cast<const double2*>(r + gi);
    const double2 qv = *reinterpret_cast<const double2*>(q + gi);
    rv.x = fma(-alpha, qv.x, rv.x);
    rv.y = fma(-alpha, qv.y, rv.y);
    if (e >= e_lo && e < e_hi) {
      if (x != nullptr) {   // null: the next p update makes it (x_lag)
        const double2 pv = *reinterpret_cast<const double2*>(p + gi);
        double2 xv = *reinterpret_cast<const double2*>(x + gi);
        xv.x = fma(alpha, pv.x, xv.x);
        xv.y = fma(alpha, pv.y, xv.y);
        *reinterpret_cast<double2*>(x + gi) = xv;
      }
      rr[0] = fma(rv.x, rv.x, rr[0]);
      rr[0] = fma(rv.y, rv.y, rr[0]);
    }
    const double2 w = *reinterpret_cast<const double2*>(wt + kp);
    acc[0] = fma(w.x, rv.x, acc[0]);
    acc[0] = fma(w.y, rv.y, acc[0]);
    store2<T>(row, kp, rv.x, rv.y, 1.0);
  }
  for (int kp = 2 * npair + 2 * threadIdx.x; kp < kpad; kp += 2 * blockDim.x) store2<T>(row, kp, 0.0, 0.0, 1.0);
  if (c0 != nullptr) {
    block_sum<1>(acc);
    if (threadIdx.x == 0) c0[s] = acc[0];
  }
  double tot[1];
  if (grid_sum_last<1>(rr, partials, counter, tot, vb) && threadIdx.x == 0) {
    const double rrv = tot[0];
    st->rr = rrv;
    st->iter += 1;
    if (!isfinite(rrv)) {
      st->status = DD_ENAN;
      st->done = 1;
    } else if (rrv <= st->tol2) {
      st->done = 1;
    } else if (st->iter >= st->maxit) {
      st->status = DD_EMAXIT;
      st->done = 1;
    }
  }
}

template <typename T>
__global__ void __launch_bounds__(128, 16) k_pack_xr(Geo g, const Sub* __restrict__ subs, const int* __restrict__ slot_of,
                                                 const double* __restrict__ r, const double* __restrict__ q,
                                                 double* __restrict__ x, double* pb0, double* pb1, int kpad,
                                                 T* __restrict__ out, const double* __restrict__ wT, double* c0,
                                                 PcgState* st, double* partials, unsigned* counter) {
  pdl_enter();
  pack_xr_body<T>(vblk_self(), g, subs, slot_of, r, q, x, pb0, pb1, kpad, out, wT, c0, st, partials, counter);
}

template <typename T>
__global__ void __launch_bounds__(128, 16) kb_pack_xr(const BInst* __restrict__ B, const int2* __restrict__ vmap) {
  const int2 m = vmap[blockIdx.x];
  const BInst& I = B[m.x];
  if (!I.active) return;
  pack_xr_body<T>(VBlk{m.y, I.nsub}, I.g, I.subs, I.slot_of_sub, I.r, I.q, I.x, I.pb0, I.pb1, I.kpad,
                         reinterpret_cast<T*>(I.Rpack), I.wT, I.coarse ? I.c0 : nullptr, I.st, I.red,
                         I.cnt + CNT_RR);
}

// one block per subdomain (blockIdx.x = subdomain id)
template <typename T>
__global__ void k_pack(Geo g, const Sub* __restrict__ subs, const int* __restrict__ slot_of,
                       const double* __restrict__ r, int kpad, T* __restrict__ out, const double* __restrict__ wT,
                       double* c0, const PcgState* st, const float* __restrict__ ascale, float* __restrict__ ysc,
                       const char* __restrict__ pf, unsigned pf_bytes) {
  pdl_enter();
  // pf: the coarse cyclic reduction's coefficients, which the iteration's other vectors have
  // pushed out of L2 since the last solve; prefetched into L2 here (a hint, nothing waits on
  // it) so that the solve that follows this pass copies them from L2 rather than from DRAM
  if (pf != nullptr && blockIdx.x == 0 && threadIdx.x == 0) {
    for (unsigned o = 0; o < pf_bytes; o += 32768u)
      asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(pf + o), "r"(min(32768u, pf_bytes - o))
                   : "memory");
  }
  pack_body<T>(g, subs, slot_of, r, kpad, out, wT, c0, st, ascale, ysc, (int)blockIdx.x);
}

// batched: vmap[blockIdx.x] = {problem, subdomain}
template <typename T>
__global__ void __launch_bounds__(128, 16) kb_pack(const BInst* __restrict__ B, const int2* __restrict__ vmap) {
  const int2 m = vmap[blockIdx.x];
  const BInst& I = B[m.x];
  if (!I.active) return;
  pack_body<T>(I.g, I.subs, I.slot_of_sub, I.r, I.kpad, reinterpret_cast<T*>(I.Rpack), I.wT,
               I.coarse ? I.c0 : nullptr, I.st, nullptr, nullptr, m.y);
}

// FP8 local inverses: per-type max |A_T^{-1}| (grid = blocks x types), then the scaled rounding
__global__ void k_type_absmax(const double* __restrict__ a, long long per_type, double* partial) {
  const int ty = blockIdx.y;
  const double* at = a + (size_t)ty * per_type;
  double m = 0.0;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < per_type;
       t += (long long)gridDim.x * blockDim.x)
    m = fmax(m, fabs(at[t]));
  __shared__ double sm[32];
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(kFull, m, o));
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) sm[wid] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) m = fmax(m, sm[w]);
    partial[(size_t)ty * gridDim.x + blockIdx.x] = fmax(sm[0], m);
  }
}

__global__ void k_type_scale(const double* __restrict__ partial, int nblk, int ntypes, double* scale,
                             float* ascale) {
  const int ty = threadIdx.x;
  if (ty >= ntypes) return;
  double m = 0.0;
  for (int b = 0; b < nblk; ++b) m = fmax(m, partial[(size_t)ty * nblk + b]);
  const double sc = m > 0.0 ? kE4M3Max / m : 1.0;
  scale[ty] = sc;
  ascale[ty] = (float)(1.0 / sc);
}

__global__ void k_quantize_e4m3(const double* __restrict__ a, long long per_type, int ntypes,
                                const double* __restrict__ scale, __nv_fp8_e4m3* out) {
  const long long total = per_type * ntypes;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x)
    out[t] = to_e4m3(a[t] * scale[t / per_type]);
}

// Three output-tile shapes, 128 x 256, 128 x 160 and 128 x 128: per output element the K
// order of the accumulation is the same in all, so the choice changes the speed, not the
// result.  128 x 160 fits the 2046 interior subdomains of the L = 2048, h = 1/32, delta = 4
// box in 13 column tiles, so that its 150 tiles make one wave on 152 SMs.
constexpr int kTileN[3] = {256, 128, 160};
inline int tile_index(int bn) { return bn == 256 ? 0 : (bn == 128 ? 1 : 2); }
struct GemmPlan {
  CUtensorMap tA, tB[3];                         // tB[i]: box of kTileN[i] rows of R
  Tile* tiles[3] = {nullptr, nullptr, nullptr};   // tiles[i]: 128 x kTileN[i] output tiles
  int ntiles[3] = {0, 0, 0};
  int cap[3] = {0, 0, 0};
  int es = 2;                                     // operand bytes: 1 E4M3, 2 BF16, 4 TF32
};

// Autotuner cache: the faster N tile per problem shape (precision, K, rows per type, subdomain
// counts per type), measured once per process.
static std::mutex g_tune_mu;
static std::map<std::string, int> g_tune_bn;

template <typename T>
static void run_gemm_t(dd_ctx* c, GemmPlan* plan, int bn, const PcgState* st, cudaStream_t s, const float* ysc) {
  const int i = tile_index(bn);
  const bool pdl = c->pdl != 0 && st != nullptr;   // inside the PCG chain
  const CUtensorMap* tB = &plan->tB[i];
  if (bn == 256)
    launch_tc<T, 256>(&plan->tA, tB, plan->tiles[i], plan->ntiles[i], c->kpad, c->kpad, c->kpad, c->Y32, c->kpad,
                      c->dev_err + 8, st, s, ysc, nullptr, pdl);
  else if (bn == 160)
    launch_tc<T, 160>(&plan->tA, tB, plan->tiles[i], plan->ntiles[i], c->kpad, c->kpad, c->kpad, c->Y32, c->kpad,
                      c->dev_err + 8, st, s, ysc, nullptr, pdl);
  else
    launch_tc<T, 128>(&plan->tA, tB, plan->tiles[i], plan->ntiles[i], c->kpad, c->kpad, c->kpad, c->Y32, c->kpad,
                      c->dev_err + 8, st, s, ysc, nullptr, pdl);
}

static void run_gemm(dd_ctx* c, GemmPlan* plan, int bn, const PcgState* st, cudaStream_t s) {
  if (plan->es == 2) run_gemm_t<__nv_bfloat16>(c, plan, bn, st, s, nullptr);
  else if (plan->es == 4) run_gemm_t<float>(c, plan, bn, st, s, nullptr);
  else run_gemm_t<__nv_fp8_e4m3>(c, plan, bn, st, s, c->ysc);
}

// time the tile shapes on the context's operands (3 launches each after one warm-up)
static int tune_bn(dd_ctx* c, GemmPlan* plan) {
  std::string key = std::to_string(plan->es) + ":" + std::to_string(c->kpad);
  for (int t = 0; t < c->ntypes; ++t) key += ":" + std::to_string(c->type_count[t]);
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune_bn.find(key);
    if (it != g_tune_bn.end()) return it->second;
  }
  cudaEvent_t e0, e1;
  DD_CUDA(cudaEventCreate(&e0));
  DD_CUDA(cudaEventCreate(&e1));
  float best = 0.0f;
  int best_bn = 256;
  for (int bn : kTileN) {
    run_gemm(c, plan, bn, nullptr, c->stream);
    DD_CUDA(cudaEventRecord(e0, c->stream));
    for (int r = 0; r < 3; ++r) run_gemm(c, plan, bn, nullptr, c->stream);
    DD_CUDA(cudaEventRecord(e1, c->stream));
    DD_CUDA(cudaEventSynchronize(e1));
    float ms = 0.0f;
    DD_CUDA(cudaEventElapsedTime(&ms, e0, e1));
    if (bn == 256 || ms < best) {
      best = ms;
      best_bn = bn;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tune_bn.emplace(key, best_bn);
  return best_bn;
}

static int prec_bytes(int precision) {
  return precision == DD_PREC_BF16 ? 2 : (precision == DD_PREC_TF32 ? 4 : 1);
}

template <typename T>
static void launch_local_inverse_t(dd_ctx* c, const int* nloc, T* out) {
  const int kpad = c->kpad;
  DD_BAND_DISPATCH(c->band, {
    // identity columns solved four (two for wide bands) to a warp where the lane-owned solve
    // allows it: its sequential steps are latency-bound, and the columns share them
    constexpr int KK = (NV == 0) ? 1 : (NV <= 4 ? 4 : 2);
    const size_t per = sizeof(float) * (size_t)KK * c->nloc_max + band_ring_bytes(c->band, sizeof(float));
    const int wpb = per <= 48 * 1024 ? 2 : 1;
    const size_t smem = per * wpb;
    const long long jobs = (long long)c->ntypes * ((c->nloc_max + KK - 1) / KK);
    const int nb = (int)((jobs + wpb - 1) / wpb);
    DD_CUDA(cudaFuncSetAttribute(k_local_inverse<T, NV, PF, KK>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 220 * 1024));
    (k_local_inverse<T, NV, PF, KK><<<nb, 32 * wpb, smem, c->stream>>>(nloc, c->nloc_max, c->band, c->bandCB32,
                                                                       c->bandRB32, c->bandInv32, c->ntypes, kpad,
                                                                       c->g.nyi, c->g.ylog, out),
     dd::note_launch());
  });
  DD_CUDA(cudaGetLastError());
}

int gemm_setup(dd_ctx* c) {
  const Geo& g = c->g;
  const int es = prec_bytes(c->grid.precision);
  const int kpad = c->kpad;
  const long long per_type = (long long)kpad * kpad;
  if (!c->Ainv) {
    c->Ainv = dev_alloc(c, (size_t)es * c->ntypes * per_type);
    c->Rpack = dev_alloc(c, (size_t)es * g.nsub * kpad);
    c->Y32 = (float*)dev_alloc(c, sizeof(float) * (size_t)g.nsub * kpad);
    if (es == 1) {
      c->ysc = (float*)dev_alloc(c, sizeof(float) * g.nsub);
      c->ascale = (float*)dev_alloc(c, sizeof(float) * c->ntypes);
      c->ascale64 = (double*)dev_alloc(c, sizeof(double) * c->ntypes);
    }
  } else {
    DD_CUDA(cudaMemsetAsync(c->Ainv, 0, (size_t)es * c->ntypes * per_type, c->stream));
  }
  // local inverses
  int* nloc = nullptr;
  DD_CUDA(cudaMallocAsync(&nloc, sizeof(int) * c->ntypes, c->stream));
  DD_CUDA(cudaMemcpyAsync(nloc, c->type_nloc, sizeof(int) * c->ntypes, cudaMemcpyHostToDevice, c->stream));
  if (es == 2) {
    launch_local_inverse_t<__nv_bfloat16>(c, nloc, (__nv_bfloat16*)c->Ainv);
  } else if (es == 4) {
    launch_local_inverse_t<float>(c, nloc, (float*)c->Ainv);
  } else {
    // FP64 inverse in a scratch, per-type scale 448 / max|A_T^{-1}|, scaled E4M3 rounding
    double* a64 = nullptr;
    DD_CUDA(cudaMallocAsync(&a64, sizeof(double) * (size_t)c->ntypes * per_type, c->stream));
    DD_CUDA(cudaMemsetAsync(a64, 0, sizeof(double) * (size_t)c->ntypes * per_type, c->stream));
    launch_local_inverse_t<double>(c, nloc, a64);
    const int nblk = 64;
    double* part = nullptr;
    DD_CUDA(cudaMallocAsync(&part, sizeof(double) * nblk * c->ntypes, c->stream));
    (k_type_absmax<<<dim3(nblk, c->ntypes), 256, 0, c->stream>>>(a64, per_type, part), dd::note_launch());
    (k_type_scale<<<1, 32, 0, c->stream>>>(part, nblk, c->ntypes, c->ascale64, c->ascale), dd::note_launch());
    (k_quantize_e4m3<<<grid_blocks(per_type * c->ntypes, 256), 256, 0, c->stream>>>(
         a64, per_type, c->ntypes, c->ascale64, (__nv_fp8_e4m3*)c->Ainv),
     dd::note_launch());
    DD_CUDA(cudaGetLastError());
    DD_CUDA(cudaFreeAsync(part, c->stream));
    DD_CUDA(cudaFreeAsync(a64, c->stream));
  }
  DD_CUDA(cudaFreeAsync(nloc, c->stream));
  // plan: tensor maps and tile list
  GemmPlan* plan = reinterpret_cast<GemmPlan*>(c->tmapA);
  if (!plan) {
    plan = new GemmPlan();
    c->tmapA = plan;
  }
  plan->es = es;
  const int BK = 128 / es;   // one 128-byte swizzle row of K
  make_tmap(&plan->tA, c->Ainv, es, kpad, (long long)c->ntypes * kpad, BK, 128);
  const int mt = (kpad + 127) / 128;
  for (int i = 0; i < 3; ++i) {
    const int bn = kTileN[i];
    make_tmap(&plan->tB[i], c->Rpack, es, kpad, g.nsub, BK, bn);
    // Tiles in launch order.  Grids of several waves go band by band (per type, one 128-row
    // band of A_T^{-1} with all its column tiles), so that the CTAs in flight share a few bands
    // in L2 instead of each wave streaming the whole inverse again (L = 64, h = 1/16: 274 ->
    // 264 us per launch); a single wave keeps the column tiles outermost (L = 2048, h = 1/32:
    // 16.1 against 17.0 us band by band).
    long long total = 0;
    for (int t = 0; t < c->ntypes; ++t) total += (long long)mt * ((c->type_count[t] + bn - 1) / bn);
    const bool bands = total > 2 * 152;
    std::vector<Tile> tl;
    if (bands) {
      // Each type band by band, and the types interleaved in proportion to their tile counts:
      // a type with few subdomains (an edge or corner of the box) still reads its whole
      // inverse for a few output columns (bound by DRAM), the many-subdomain interior type is
      // bound by the tensor pipe, and spread through the launch order the two kinds of tiles
      // run side by side instead of one phase after the other.
      std::vector<std::pair<double, Tile>> keyed;
      for (int t = 0; t < c->ntypes; ++t) {
        const int first = c->type_first[t], cnt = c->type_count[t];
        const int nt = mt * ((cnt + bn - 1) / bn);
        int i = 0;
        for (int m = 0; m < mt; ++m)
          for (int n0 = 0; n0 < cnt; n0 += bn, ++i)
            keyed.push_back({(i + 0.5) / nt, Tile{t, m * 128, first + n0, first + cnt}});
      }
      std::stable_sort(keyed.begin(), keyed.end(),
                       [](const std::pair<double, Tile>& a, const std::pair<double, Tile>& b) { return a.first < b.first; });
      for (const auto& k : keyed) tl.push_back(k.second);
    } else {
      for (int t = 0; t < c->ntypes; ++t) {
        const int first = c->type_first[t], cnt = c->type_count[t];
        for (int n0 = 0; n0 < cnt; n0 += bn)
          for (int m = 0; m < mt; ++m) tl.push_back(Tile{t, m * 128, first + n0, first + cnt});
      }
    }
    if (!plan->tiles[i] || plan->cap[i] < (int)tl.size()) {
      plan->tiles[i] = (Tile*)dev_alloc(c, sizeof(Tile) * tl.size());
      plan->cap[i] = (int)tl.size();
    }
    plan->ntiles[i] = (int)tl.size();
    DD_CUDA(cudaMemcpyAsync(plan->tiles[i], tl.data(), sizeof(Tile) * tl.size(), cudaMemcpyHostToDevice, c->stream));
  }
  DD_CUDA(cudaStreamSynchronize(c->stream));
  if (c->gemm_bn == 0) c->gemm_bn = c->gemm_bn_opt != 0 ? c->gemm_bn_opt : tune_bn(c, plan);
  c->gemm_ok = 1;
  return DD_OK;
}

// 128 threads (16 blocks of 31 registers per SM): all 2048 subdomain blocks of the
// L = 2048, h = 1/32 box are resident at once instead of 1216 + 832 blocks of 256 (14.3
// against 15.6 us)
constexpr int kPackThreads = 128;

void launch_pack(dd_ctx* c, const double* r, double* c0, cudaStream_t s) {
  const Geo& g = c->g;
  const bool pdl = c->pdl != 0;
  const PcgState* st = c->st;
  // the staged part of the cyclic reduction's coefficients (a multiple of 16 bytes)
  const bool pf_on = c0 != nullptr && !c->coarse_dense && c->cr != nullptr;
  const char* pf = pf_on ? reinterpret_cast<const char*>(c->cr) : nullptr;
  const unsigned pf_bytes = pf_on ? (unsigned)(sizeof(double) * (2 * (size_t)c->cr_c2 + 3 * (size_t)c->cr_w2)) : 0u;
  if (c->grid.precision == DD_PREC_BF16)
    launch_chain(k_pack<__nv_bfloat16>, dim3(g.nsub), dim3(kPackThreads), 0, s, pdl, g, (const Sub*)c->subs,
                 (const int*)c->slot_of_sub, r, c->kpad, (__nv_bfloat16*)c->Rpack, (const double*)c->wT, c0, st,
                 (const float*)nullptr, (float*)nullptr, pf, pf_bytes);
  else if (c->grid.precision == DD_PREC_TF32)
    launch_chain(k_pack<float>, dim3(g.nsub), dim3(kPackThreads), 0, s, pdl, g, (const Sub*)c->subs,
                 (const int*)c->slot_of_sub, r, c->kpad, (float*)c->Rpack, (const double*)c->wT, c0, st,
                 (const float*)nullptr, (float*)nullptr, pf, pf_bytes);
  else
    launch_chain(k_pack<__nv_fp8_e4m3>, dim3(g.nsub), dim3(kPackThreads), 0, s, pdl, g, (const Sub*)c->subs,
                 (const int*)c->slot_of_sub, r, c->kpad, (__nv_fp8_e4m3*)c->Rpack, (const double*)c->wT, c0, st,
                 (const float*)c->ascale, (float*)c->ysc, pf, pf_bytes);
}

void launch_pack_xr(dd_ctx* c, cudaStream_t s) {
  const Geo& g = c->g;
  const bool pdl = c->pdl != 0;
  double* c0 = c->grid.coarse ? c->c0 : nullptr;
#define DD_PACK_XR(T)                                                                                           \
  launch_chain(k_pack_xr<T>, dim3(g.nsub), dim3(kPackThreads), 0, s, pdl, g, (const Sub*)c->subs,             \
               (const int*)c->slot_of_sub, (const double*)c->r, (const double*)c->q,                              \
               x_lag_target(c) != nullptr ? nullptr : c->x, c->pb[0], c->pb[1],                                 \
               c->kpad, (T*)c->Rpack, (const double*)c->wT, c0, c->st, c->red, c->cnt + CNT_RR)
  if (c->grid.precision == DD_PREC_BF16) {
    DD_PACK_XR(__nv_bfloat16);
  } else if (c->grid.precision == DD_PREC_TF32) {
    DD_PACK_XR(float);
  } else {
    throw Error(DD_EUNSUPPORTED, "the fused x/r update and packing takes BF16 or TF32 operands");
  }
#undef DD_PACK_XR
}

int launch_gemm(dd_ctx* c, cudaStream_t s) {
  GemmPlan* plan = reinterpret_cast<GemmPlan*>(c->tmapA);
  if (!c->gemm_ok || !plan) return DD_ESTATE;
  run_gemm(c, plan, c->gemm_bn_opt != 0 ? c->gemm_bn_opt : c->gemm_bn, c->st, s);
  return DD_OK;
}

void gemm_free(dd_ctx* c) {
  delete reinterpret_cast<GemmPlan*>(c->tmapA);
  c->tmapA = nullptr;
}

void launch_b_pack_xr(const BInst* B, const int2* vmap, int nvb, int precision, cudaStream_t s) {
  if (precision == DD_PREC_BF16) {
    (kb_pack_xr<__nv_bfloat16><<<nvb, kPackThreads, 0, s>>>(B, vmap), dd::note_launch());
  } else if (precision == DD_PREC_TF32) {
    (kb_pack_xr<float><<<nvb, kPackThreads, 0, s>>>(B, vmap), dd::note_launch());
  } else {
    throw Error(DD_EUNSUPPORTED, "batched packing supports BF16 and TF32 operands");
  }
  DD_CUDA(cudaGetLastError());
}

void launch_b_pack(const BInst* B, const int2* vmap, int nvb, int precision, cudaStream_t s) {
  if (precision == DD_PREC_BF16)
    (kb_pack<__nv_bfloat16><<<nvb, kPackThreads, 0, s>>>(B, vmap), dd::note_launch());
  else if (precision == DD_PREC_TF32)
    (kb_pack<float><<<nvb, kPackThreads, 0, s>>>(B, vmap), dd::note_launch());
  else
    throw Error(DD_EUNSUPPORTED, "batched packing supports BF16 and TF32 operands");
  DD_CUDA(cudaGetLastError());
}

// ----------------------------------------------------------------------------------------
// Grouped local-solve contraction of a batch: the problems' rounded inverses, packed
// restrictions and local solutions live in three batch-wide buffers (problem i's rows
// start at type_base[i] kpad, slot_base[i] and slot_base[i] rows), so one pair of tensor
// maps and one tile list cover every problem, and each tile carries its problem's PCG state
// (its CTAs return at once when that problem's solve is done).  Per output element the K
// order of the accumulation is that of the problem's own launch: results are identical.
// ----------------------------------------------------------------------------------------
struct BGemm {
  CUtensorMap tA, tB[3];
  Tile* tiles[3] = {nullptr, nullptr, nullptr};
  const PcgState** tile_st[3] = {nullptr, nullptr, nullptr};
  int ntiles[3] = {0, 0, 0};
  int es = 2, kpad = 0, bn = 0;
  float* Y = nullptr;
  int* err = nullptr;
};

BGemm* bgemm_create(const std::vector<dd_ctx*>& cs, const std::vector<int>& type_base,
                    const std::vector<int>& slot_base, void* Ainv_all, void* Rpack_all, float* Y_all, int* err,
                    cudaStream_t s) {
  BGemm* b = new BGemm();
  try {
    const dd_ctx* c0 = cs.front();
    b->es = prec_bytes(c0->grid.precision);
    b->kpad = c0->kpad;
    b->Y = Y_all;
    b->err = err;
    int types = 0, slots = 0;
    for (size_t i = 0; i < cs.size(); ++i) {
      types = std::max(types, type_base[i] + cs[i]->ntypes);
      slots = std::max(slots, slot_base[i] + cs[i]->g.nsub);
    }
    const int BK = 128 / b->es;
    make_tmap(&b->tA, Ainv_all, b->es, b->kpad, (long long)types * b->kpad, BK, 128);
    const int mt = (b->kpad + 127) / 128;
    for (int k = 0; k < 3; ++k) {
      const int bn = kTileN[k];
      make_tmap(&b->tB[k], Rpack_all, b->es, b->kpad, slots, BK, bn);
      std::vector<Tile> tl;
      std::vector<const PcgState*> ts;
      for (size_t i = 0; i < cs.size(); ++i) {
        const dd_ctx* c = cs[i];
        for (int t = 0; t < c->ntypes; ++t) {
          const int first = slot_base[i] + c->type_first[t], cnt = c->type_count[t];
          for (int n0 = 0; n0 < cnt; n0 += bn)
            for (int m = 0; m < mt; ++m) {
              tl.push_back(Tile{type_base[i] + t, m * 128, first + n0, first + cnt});
              ts.push_back(c->st);
            }
        }
      }
      DD_CUDA(cudaMalloc(&b->tiles[k], sizeof(Tile) * tl.size()));
      DD_CUDA(cudaMalloc(&b->tile_st[k], sizeof(PcgState*) * ts.size()));
      DD_CUDA(cudaMemcpyAsync(b->tiles[k], tl.data(), sizeof(Tile) * tl.size(), cudaMemcpyHostToDevice, s));
      DD_CUDA(cudaMemcpyAsync(b->tile_st[k], ts.data(), sizeof(PcgState*) * ts.size(), cudaMemcpyHostToDevice, s));
      b->ntiles[k] = (int)tl.size();
    }
    DD_CUDA(cudaStreamSynchronize(s));
  } catch (...) {
    bgemm_destroy(b);
    throw;
  }
  return b;
}

void bgemm_destroy(BGemm* b) {
  if (!b) return;
  for (int k = 0; k < 3; ++k) {
    if (b->tiles[k]) cudaFree(b->tiles[k]);
    if (b->tile_st[k]) cudaFree(b->tile_st[k]);
  }
  delete b;
}

template <typename T>
static void bgemm_run_t(BGemm* b, int bn, cudaStream_t s) {
  const int k = tile_index(bn);
  if (bn == 256)
    launch_tc<T, 256>(&b->tA, &b->tB[k], b->tiles[k], b->ntiles[k], b->kpad, b->kpad, b->kpad, b->Y, b->kpad, b->err,
                      nullptr, s, nullptr, b->tile_st[k]);
  else if (bn == 160)
    launch_tc<T, 160>(&b->tA, &b->tB[k], b->tiles[k], b->ntiles[k], b->kpad, b->kpad, b->kpad, b->Y, b->kpad, b->err,
                      nullptr, s, nullptr, b->tile_st[k]);
  else
    launch_tc<T, 128>(&b->tA, &b->tB[k], b->tiles[k], b->ntiles[k], b->kpad, b->kpad, b->kpad, b->Y, b->kpad, b->err,
                      nullptr, s, nullptr, b->tile_st[k]);
}

void bgemm_run(BGemm* b, int bn, cudaStream_t s) {
  if (b->es == 2) bgemm_run_t<__nv_bfloat16>(b, bn, s);
  else if (b->es == 4) bgemm_run_t<float>(b, bn, s);
  else throw Error(DD_EUNSUPPORTED, "grouped contraction supports BF16 and TF32 operands");
}

// the N tile of the grouped launch, by timing each shape on the batch's operands; every tile
// reads its problem's PCG state, so the caller clears the done flags first
int bgemm_tune(BGemm* b, cudaStream_t s) {
  cudaEvent_t e0, e1;
  DD_CUDA(cudaEventCreate(&e0));
  DD_CUDA(cudaEventCreate(&e1));
  float best = 0.0f;
  int best_bn = 256;
  try {
    for (int bn : kTileN) {
      bgemm_run(b, bn, s);
      DD_CUDA(cudaEventRecord(e0, s));
      for (int r = 0; r < 3; ++r) bgemm_run(b, bn, s);
      DD_CUDA(cudaEventRecord(e1, s));
      DD_CUDA(cudaEventSynchronize(e1));
      float ms = 0.0f;
      DD_CUDA(cudaEventElapsedTime(&ms, e0, e1));
      if (bn == 256 || ms < best) {
        best = ms;
        best_bn = bn;
      }
    }
  } catch (...) {
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    throw;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  b->bn = best_bn;
  return best_bn;
}

}  // namespace dd

// ------------------------------------------------------------------------------------------
// Diagnostic entry point: D[n][m] = sum_k A[m][k] B[n][k] through the same kernel.
// ------------------------------------------------------------------------------------------
namespace dd {

// E4M3 bits of a float (1 sign, 4 exponent bits with bias 7, 3 mantissa bits, subnormals below
// 2^-6, no infinities; nearest even, saturating at 448), from the format's definition
static uint8_t host_e4m3(float f) {
  const uint8_t sign = std::signbit(f) ? 0x80 : 0x00;
  double a = std::fabs((double)f);
  if (a == 0.0) return sign;
  if (a >= 448.0) return sign | 0x7E;
  int e;
  std::frexp(a, &e);   // a = fr 2^e, fr in [0.5, 1): exponent of the leading bit is e - 1
  int E = e - 1;
  if (E < -6) {        // subnormal: units of 2^-9
    const double q = a * 512.0;
    double m = std::nearbyint(q);
    if (m >= 8.0) return sign | (1u << 3);   // rounds up to the smallest normal
    return sign | (uint8_t)m;
  }
  double mant = a / std::ldexp(1.0, E) - 1.0;   // in [0, 1)
  double m = std::nearbyint(mant * 8.0);
  if (m >= 8.0) {
    m = 0.0;
    ++E;
  }
  if (E > 8 || (E == 8 && m > 6.0)) return sign | 0x7E;
  return sign | (uint8_t)(((E + 7) << 3) | (int)m);
}

}  // namespace dd

namespace dd {
constexpr int kTestMaxDim = 1 << 16;   // largest M, N or K accepted by dd_tc_gemm_test
}

extern "C" int dd_tc_gemm_test(int precision, int M, int N, int K, const float* A_host, const float* B_host,
                               float* D_host) {
  using namespace dd;
  if (precision != DD_PREC_BF16 && precision != DD_PREC_TF32 && precision != DD_PREC_FP8) return DD_EINVAL;
  if (M < 1 || N < 1 || K < 1 || !A_host || !B_host || !D_host) return DD_EINVAL;
  // a self-test stages whole host copies of its operands: sizes stay far below int overflow
  if (M > kTestMaxDim || N > kTestMaxDim || K > kTestMaxDim) return DD_EINVAL;
  const int es = precision == DD_PREC_BF16 ? 2 : (precision == DD_PREC_TF32 ? 4 : 1);
  const int kpad = (K + 127) / 128 * 128;
  const int mpad = (M + 127) / 128 * 128;
  void *dA = nullptr, *dB = nullptr;
  float* dD = nullptr;
  int* derr = nullptr;
  Tile* dt = nullptr;
  cudaStream_t s = nullptr;
  int rc = DD_OK;
  try {
    DD_CUDA(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
    DD_CUDA(cudaMalloc(&dA, (size_t)es * mpad * kpad));
    DD_CUDA(cudaMalloc(&dB, (size_t)es * N * kpad));
    DD_CUDA(cudaMalloc(&dD, sizeof(float) * (size_t)N * mpad));
    DD_CUDA(cudaMalloc(&derr, sizeof(int)));
    DD_CUDA(cudaMemsetAsync(derr, 0, sizeof(int), s));
    // operands rounded on the host: BF16 and E4M3 to nearest even, TF32 passed as FP32
    std::vector<uint8_t> a8, b8;
    std::vector<uint16_t> a16, b16;
    std::vector<float> a32, b32;
    auto to_bf16 = [](float f) -> uint16_t {
      uint32_t u;
      std::memcpy(&u, &f, 4);
      const uint32_t lsb = (u >> 16) & 1u;
      u += 0x7FFFu + lsb;
      return (uint16_t)(u >> 16);
    };
    if (es == 2) {
      a16.assign((size_t)mpad * kpad, 0);
      b16.assign((size_t)N * kpad, 0);
      for (int m = 0; m < M; ++m)
        for (int k = 0; k < K; ++k) a16[(size_t)m * kpad + k] = to_bf16(A_host[(size_t)m * K + k]);
      for (int n = 0; n < N; ++n)
        for (int k = 0; k < K; ++k) b16[(size_t)n * kpad + k] = to_bf16(B_host[(size_t)n * K + k]);
      DD_CUDA(cudaMemcpyAsync(dA, a16.data(), a16.size() * 2, cudaMemcpyHostToDevice, s));
      DD_CUDA(cudaMemcpyAsync(dB, b16.data(), b16.size() * 2, cudaMemcpyHostToDevice, s));
    } else if (es == 1) {
      a8.assign((size_t)mpad * kpad, 0);
      b8.assign((size_t)N * kpad, 0);
      for (int m = 0; m < M; ++m)
        for (int k = 0; k < K; ++k) a8[(size_t)m * kpad + k] = host_e4m3(A_host[(size_t)m * K + k]);
      for (int n = 0; n < N; ++n)
        for (int k = 0; k < K; ++k) b8[(size_t)n * kpad + k] = host_e4m3(B_host[(size_t)n * K + k]);
      DD_CUDA(cudaMemcpyAsync(dA, a8.data(), a8.size(), cudaMemcpyHostToDevice, s));
      DD_CUDA(cudaMemcpyAsync(dB, b8.data(), b8.size(), cudaMemcpyHostToDevice, s));
    } else {
      a32.assign((size_t)mpad * kpad, 0.f);
      b32.assign((size_t)N * kpad, 0.f);
      for (int m = 0; m < M; ++m)
        for (int k = 0; k < K; ++k) a32[(size_t)m * kpad + k] = A_host[(size_t)m * K + k];
      for (int n = 0; n < N; ++n)
        for (int k = 0; k < K; ++k) b32[(size_t)n * kpad + k] = B_host[(size_t)n * K + k];
      DD_CUDA(cudaMemcpyAsync(dA, a32.data(), a32.size() * 4, cudaMemcpyHostToDevice, s));
      DD_CUDA(cudaMemcpyAsync(dB, b32.data(), b32.size() * 4, cudaMemcpyHostToDevice, s));
    }
    CUtensorMap tA, tB;
    const int BK = 128 / es;
    make_tmap(&tA, dA, es, kpad, mpad, BK, 128);
    make_tmap(&tB, dB, es, kpad, N, BK, 256);
    std::vector<Tile> tl;
    for (int n0 = 0; n0 < N; n0 += 256)
      for (int m0 = 0; m0 < mpad; m0 += 128) tl.push_back(Tile{0, m0, n0, N});
    DD_CUDA(cudaMalloc(&dt, sizeof(Tile) * tl.size()));
    DD_CUDA(cudaMemcpyAsync(dt, tl.data(), sizeof(Tile) * tl.size(), cudaMemcpyHostToDevice, s));
    if (es == 2)
      launch_tc<__nv_bfloat16>(&tA, &tB, dt, (int)tl.size(), kpad, mpad, 0, dD, mpad, derr, nullptr, s);
    else if (es == 4)
      launch_tc<float>(&tA, &tB, dt, (int)tl.size(), kpad, mpad, 0, dD, mpad, derr, nullptr, s);
    else
      launch_tc<__nv_fp8_e4m3>(&tA, &tB, dt, (int)tl.size(), kpad, mpad, 0, dD, mpad, derr, nullptr, s);
    std::vector<float> hD((size_t)N * mpad);
    int herr = 0;
    DD_CUDA(cudaMemcpyAsync(hD.data(), dD, sizeof(float) * hD.size(), cudaMemcpyDeviceToHost, s));
    DD_CUDA(cudaMemcpyAsync(&herr, derr, sizeof(int), cudaMemcpyDeviceToHost, s));
    DD_CUDA(cudaStreamSynchronize(s));
    for (int n = 0; n < N; ++n)
      for (int m = 0; m < M; ++m) D_host[(size_t)n * M + m] = hD[(size_t)n * mpad + m];
    if (herr) rc = DD_ETIMEOUT;
  } catch (const Error& e) {
    rc = e.code;
  } catch (const std::bad_alloc&) {
    rc = DD_ENOMEM;
  }
  if (dA) cudaFree(dA);
  if (dB) cudaFree(dB);
  if (dD) cudaFree(dD);
  if (derr) cudaFree(derr);
  if (dt) cudaFree(dt);
  if (s) cudaStreamDestroy(s);
  return rc;
}

// ------------------------------------------------------------------------------------------
// Allocation-free variant of the tensor-core contraction.
//
// Some callers cannot allocate device memory at the point where they need this product:
// a serving process that reserves all device memory in its own arena at start-up (a
// cudaMalloc from inside the request path would fail or fragment that arena), code on a
// latency-critical path where cudaMalloc/cudaFree would synchronise the device, or code
// running under another framework's memory manager that forbids raw allocations.  For
// them this entry point takes device operands and a device output and keeps the kernel's
// scratch (the tile list and the error word of its bounded waits) in a fixed array that
// lives in this library's static device memory: kNoAllocBytes bytes on every GPU that
// loads the library, held until the process exits.
// ------------------------------------------------------------------------------------------
#include <mutex>

namespace dd {

constexpr int kNoAllocMaxTiles = 4096;                          // 128 x 256 output tiles
constexpr size_t kNoAllocBytes = 256 + sizeof(Tile) * kNoAllocMaxTiles;   // 64 KB + error word

// [0, 256): error word (int); [256, ...): tile list
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

static std::mutex g_noalloc_mu;
static void* g_noalloc_addr[256];   // device address of g_noalloc_scratch, per device ordinal

// Resolves the device address of the scratch array for the current device (once per device).
static int noalloc_scratch(void** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 256) return DD_ECUDA;
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (!g_noalloc_addr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || p == nullptr) {
      cudaGetLastError();
      return DD_ECUDA;
    }
    g_noalloc_addr[dev] = p;
  }
  *out = g_noalloc_addr[dev];
  return DD_OK;
}

}  // namespace dd

extern "C" int dd_tc_gemm_noalloc(int precision, int M, int N, int K, const void* A_dev, const void* B_dev,
                                  float* D_dev, void* stream) {
  using namespace dd;
  if (precision != DD_PREC_BF16 && precision != DD_PREC_TF32) return DD_EINVAL;
  if (M < 1 || N < 1 || K < 64 || (K % 64) != 0 || !A_dev || !B_dev || !D_dev) return DD_EINVAL;
  // tile count in 64-bit arithmetic: M + 127 or N + 255 would overflow int near INT_MAX
  const long long ntiles = (((long long)M + 127) / 128) * (((long long)N + 255) / 256);
  if (ntiles > kNoAllocMaxTiles) return DD_EINVAL;   // output larger than the fixed scratch allows
  void* scratch = nullptr;
  int rc = noalloc_scratch(&scratch);
  if (rc != DD_OK) return rc;
  int* derr = reinterpret_cast<int*>(scratch);
  Tile* dtiles = reinterpret_cast<Tile*>(reinterpret_cast<unsigned char*>(scratch) + 256);
  cudaStream_t s = (cudaStream_t)stream;
  try {
    const bool bf16 = precision == DD_PREC_BF16;
    Tile tl[kNoAllocMaxTiles];
    int nt = 0;
    for (int n0 = 0; n0 < N; n0 += 256)
      for (int m0 = 0; m0 < M; m0 += 128) tl[nt++] = Tile{0, m0, n0, N};
    CUtensorMap tA, tB;
    const int BK = bf16 ? TcCfg<__nv_bfloat16>::BK : TcCfg<float>::BK;
    make_tmap(&tA, const_cast<void*>(A_dev), bf16 ? 2 : 4, K, M, BK, 128);
    make_tmap(&tB, const_cast<void*>(B_dev), bf16 ? 2 : 4, K, N, BK, 256);
    // the error word must start at zero; the tile list is rewritten whole on every call
    DD_CUDA(cudaMemsetAsync(derr, 0, sizeof(int), s));
    DD_CUDA(cudaMemcpyAsync(dtiles, tl, sizeof(Tile) * nt, cudaMemcpyHostToDevice, s));
    if (bf16)
      launch_tc<__nv_bfloat16>(&tA, &tB, dtiles, nt, K, M, 0, D_dev, M, derr, nullptr, s);
    else
      launch_tc<float>(&tA, &tB, dtiles, nt, K, M, 0, D_dev, M, derr, nullptr, s);
    int herr = 0;
    DD_CUDA(cudaMemcpyAsync(&herr, derr, sizeof(int), cudaMemcpyDeviceToHost, s));
    DD_CUDA(cudaStreamSynchronize(s));
    if (herr) return DD_ETIMEOUT;
  } catch (const Error& e) {
    return e.code;
  }
  return DD_OK;
}
