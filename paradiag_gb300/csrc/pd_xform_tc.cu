// x-eigentransform of the mixed-precision path on the 5th-generation tensor
// cores (tcgen05, TMEM accumulators, TMA operand loads).
//
// Every row r of the half spectrum (one per time frequency k and grid line y)
// holds nx complex values X[r][x]; the transform is Y[r][j] = sum_x Q[j][x] X[r][x]
// with Q the eigenvector matrix of K_x (DFT for periodic x, sine transform for
// symmetric Dirichlet x).  In real form, with the interleaved (re, im) storage
// read as a row of 2nx reals, it is the GEMM
//     D[r][n] = sum_k A[r][k] G[n][k],   A = spectrum rows, G = real form of Q,
// with M = rows, N = K = 2nx, both operands K-major.
//
// Precision: split TF32 ("3xTF32").  A = A_hi + A_lo with A_hi the FP32 value
// with its 13 low significand bits cleared and A_lo = A - A_hi (exact), and the
// same for G (split on the host).  D = A_hi G_hi + A_hi G_lo + A_lo G_hi with
// FP32 accumulation, a relative error of about 2^-21, comparable to an FP32
// GEMM.  A is split in shared memory after its TMA load (the split is
// elementwise, so it does not depend on the swizzled layout).
//
// CTA tile 128 x 256 (M x N), K chunks of 32 (one 128-byte swizzle row),
// two pipeline stages.  Warp roles: warp 0 issues TMA loads, warp 1 allocates
// TMEM and issues the MMAs (one elected thread), warps 2-5 split A and then
// drain the accumulator (tcgen05.ld) to global memory.  Every mbarrier wait is
// bounded; on a timeout the CTA records an error bit, drains, frees its TMEM and
// returns.
#include <cuda.h>

#include "pd_internal.h"
#include "pd_xform_tc.h"

namespace {

constexpr int BM = 128, BN = 256, BK = 32;
constexpr int STAGES = 2;
constexpr int A_BYTES = BM * BK * 4;   // 16 KB
constexpr int B_BYTES = BN * BK * 4;   // 32 KB
constexpr int STAGE_BYTES = 2 * A_BYTES + 2 * B_BYTES;
constexpr int TMEM_COLS = 256;
constexpr int NTHREADS = 192;
constexpr long long WAIT_LIMIT = 1LL << 22;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t phase) {
  uint32_t ok;
  asm volatile(
      "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      "selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(bar), "r"(phase)
      : "memory");
  return ok != 0;
}
// bounded wait; returns false (and raises the CTA abort flag) on timeout
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t phase, volatile int* abort_flag) {
  for (long long i = 0; i < WAIT_LIMIT; ++i) {
    if (mbar_try(bar, phase)) return true;
    if ((i & 255) == 255 && *abort_flag) return false;
  }
  *abort_flag = 1;
  return false;
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, int c0, int c1,
                                            uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, "
      "%3}], [%4];" ::"r"(dst),
      "l"(map), "r"(c0), "r"(c1), "r"(bar)
      : "memory");
}

// shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups
// 1024 bytes apart (tcgen05 descriptor format: start >> 4 in bits 0-13, leading
// offset >> 4 in 16-29, stride offset >> 4 in 32-45, version 1 in 46-47,
// swizzle mode in 61-63 with 2 = 128-byte swizzle)
__device__ __forceinline__ uint64_t sdesc(uint32_t addr) {
  uint64_t d = 0;
  d |= (uint64_t)((addr & 0x3FFFF) >> 4);
  d |= (uint64_t)1 << 16;
  d |= (uint64_t)(1024 >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)2 << 61;
  return d;
}

// instruction descriptor of kind::tf32: D f32 (bits 4-5 = 1), A and B tf32
// (bits 7-9 and 10-12 = 2), both K-major, N >> 3 in bits 17-22, M >> 4 in 24-28
constexpr uint32_t IDESC = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(BN >> 3) << 17) |
                           ((uint32_t)(BM >> 4) << 24);

__device__ __forceinline__ void mma_tf32(uint32_t tmem, uint64_t a, uint64_t b, uint32_t acc) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}" ::"r"(tmem),
      "l"(a), "l"(b), "r"(IDESC), "r"(acc)
      : "memory");
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
      : "memory");
}

__global__ void __launch_bounds__(NTHREADS, 1)
    k_xform_tc(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmBhi,
               const __grid_constant__ CUtensorMap tmBlo, float* __restrict__ out, int rows,
               int ncols, int ldo, int kchunks, int* err) {
  extern __shared__ __align__(1024) unsigned char smraw[];
  // 1024-byte aligned operand stages (required by the 128-byte swizzle)
  unsigned char* base = (unsigned char*)(((uintptr_t)smraw + 1023) & ~(uintptr_t)1023);
  __shared__ __align__(8) uint64_t bar_full[STAGES], bar_split[STAGES], bar_empty[STAGES], bar_acc;
  __shared__ uint32_t tmem_slot;
  __shared__ int abort_flag;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int r0 = blockIdx.x * BM, n0 = blockIdx.y * BN;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(smem_u32(&bar_full[s]), 1);
      mbar_init(smem_u32(&bar_split[s]), 4);
      mbar_init(smem_u32(&bar_empty[s]), 1);
    }
    mbar_init(smem_u32(&bar_acc), 1);
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&tmem_slot)),
                 "r"(TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_slot;
  volatile int* abortp = &abort_flag;

  auto stage_ptr = [&](int s, int which) -> unsigned char* {
    // which: 0 A_hi (raw A loaded here), 1 A_lo, 2 B_hi, 3 B_lo
    const int off[4] = {0, A_BYTES, 2 * A_BYTES, 2 * A_BYTES + B_BYTES};
    return base + (size_t)s * STAGE_BYTES + off[which];
  };

  if (warp == 0) {
    // ---------------- TMA producer
    if (lane == 0) {
      int issued = 0;
      for (int c = 0; c < kchunks; ++c) {
        const int s = c % STAGES;
        const uint32_t ph = (uint32_t)((c / STAGES) & 1);
        if (c >= STAGES && !mbar_wait(smem_u32(&bar_empty[s]), ph ^ 1u, abortp)) break;
        const uint32_t fb = smem_u32(&bar_full[s]);
        mbar_expect_tx(fb, (uint32_t)(A_BYTES + 2 * B_BYTES));
        tma_load_2d(smem_u32(stage_ptr(s, 0)), &tmA, c * BK, r0, fb);
        tma_load_2d(smem_u32(stage_ptr(s, 2)), &tmBhi, c * BK, n0, fb);
        tma_load_2d(smem_u32(stage_ptr(s, 3)), &tmBlo, c * BK, n0, fb);
        issued = c + 1;
      }
      // drain: wait for the loads still in flight before the CTA may exit
      for (int c = (issued > STAGES ? issued - STAGES : 0); c < issued; ++c)
        mbar_wait(smem_u32(&bar_full[c % STAGES]), (uint32_t)((c / STAGES) & 1), abortp);
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer
    if (lane == 0) {
      bool ok = true;
      for (int c = 0; c < kchunks && ok; ++c) {
        const int s = c % STAGES;
        const uint32_t ph = (uint32_t)((c / STAGES) & 1);
        if (!mbar_wait(smem_u32(&bar_split[s]), ph, abortp)) { ok = false; break; }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t ahi = smem_u32(stage_ptr(s, 0)), alo = smem_u32(stage_ptr(s, 1));
        const uint32_t bhi = smem_u32(stage_ptr(s, 2)), blo = smem_u32(stage_ptr(s, 3));
#pragma unroll
        for (int kk = 0; kk < BK / 8; ++kk) {
          const uint32_t koff = kk * 32;  // 8 tf32 = 32 bytes along the swizzled row
          const uint32_t first = (c == 0 && kk == 0) ? 0u : 1u;
          mma_tf32(tmem, sdesc(ahi + koff), sdesc(bhi + koff), first);
          mma_tf32(tmem, sdesc(ahi + koff), sdesc(blo + koff), 1u);
          mma_tf32(tmem, sdesc(alo + koff), sdesc(bhi + koff), 1u);
        }
        mma_commit(smem_u32(&bar_empty[s]));
      }
      mma_commit(smem_u32(&bar_acc));
    }
  } else {
    // ---------------- A split (warps 2-5), then the epilogue
    const int t = threadIdx.x - 64;  // 0..127
    for (int c = 0; c < kchunks; ++c) {
      const int s = c % STAGES;
      const uint32_t ph = (uint32_t)((c / STAGES) & 1);
      if (!mbar_wait(smem_u32(&bar_full[s]), ph, abortp)) break;
      float4* hi = reinterpret_cast<float4*>(stage_ptr(s, 0));
      float4* lo = reinterpret_cast<float4*>(stage_ptr(s, 1));
#pragma unroll
      for (int q = 0; q < A_BYTES / 16 / 128; ++q) {
        const int i = t + q * 128;
        float4 v = hi[i], h, l;
        h.x = __uint_as_float(__float_as_uint(v.x) & 0xFFFFE000u);
        h.y = __uint_as_float(__float_as_uint(v.y) & 0xFFFFE000u);
        h.z = __uint_as_float(__float_as_uint(v.z) & 0xFFFFE000u);
        h.w = __uint_as_float(__float_as_uint(v.w) & 0xFFFFE000u);
        l.x = v.x - h.x; l.y = v.y - h.y; l.z = v.z - h.z; l.w = v.w - h.w;
        hi[i] = h;
        lo[i] = l;
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      __syncwarp();
      if (lane == 0) mbar_arrive(smem_u32(&bar_split[s]));
    }
    // epilogue: TMEM lanes 32*(warp % 4) .. +31 hold rows r0 + that range
    const bool acc_ok = mbar_wait(smem_u32(&bar_acc), 0u, abortp);
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const int q4 = warp & 3;
    const int row = r0 + q4 * 32 + lane;
    if (acc_ok) {
      for (int j = 0; j < BN; j += 16) {
        uint32_t v[16];
        const uint32_t taddr = tmem + ((uint32_t)(q4 * 32) << 16) + (uint32_t)j;
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,"
            "%13,%14,%15}, [%16];"
            : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
              "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]),
              "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
            : "r"(taddr));
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        const int n = n0 + j;
        if (row < rows) {
          float* o = out + (size_t)row * ldo + n;
          if (n + 16 <= ncols) {
#pragma unroll
            for (int u = 0; u < 4; ++u)
              reinterpret_cast<float4*>(o)[u] =
                  make_float4(__uint_as_float(v[4 * u]), __uint_as_float(v[4 * u + 1]),
                              __uint_as_float(v[4 * u + 2]), __uint_as_float(v[4 * u + 3]));
          } else {
#pragma unroll
            for (int u = 0; u < 16; ++u)
              if (n + u < ncols) o[u] = __uint_as_float(v[u]);
          }
        }
      }
    }
  }

  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 1) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(TMEM_COLS)
                 : "memory");
  }
  if (threadIdx.x == 0 && abort_flag && err != nullptr) atomicOr(err, 2);
}

// cuTensorMapEncodeTiled through the runtime's driver entry point (no link
// against the driver library)
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                  const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                  const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (EncodeTiledFn)p;
  }
  return fn;
}

bool encode_2d(CUtensorMap* m, const void* ptr, uint64_t inner, uint64_t outer,
               uint64_t row_bytes, uint32_t box_inner, uint32_t box_outer) {
  EncodeTiledFn fn = encode_fn();
  if (!fn) return false;
  const cuuint64_t dims[2] = {inner, outer};
  const cuuint64_t strides[1] = {row_bytes};
  const cuuint32_t box[2] = {box_inner, box_outer};
  const cuuint32_t estr[2] = {1, 1};
  return fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<void*>(ptr), dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace

size_t xform_tc_bpad(int nx) { return (size_t)(((2 * nx + BN - 1) / BN) * BN); }

cudaError_t xform_tc_prepare(XformTc* x, int rows, int nx, int ldo_floats, const float* in,
                             float* out, const float* Bhi, const float* Blo) {
  const uint64_t K2 = 2 * (uint64_t)nx;
  const uint64_t P = xform_tc_bpad(nx);
  x->rows = rows;
  x->ncols = (int)K2;
  x->ldo = ldo_floats;
  x->kchunks = (int)((K2 + BK - 1) / BK);
  x->nblk_n = (int)(P / BN);
  x->out = out;
  if ((ldo_floats * 4) % 16 != 0) return cudaErrorInvalidValue;
  if (!encode_2d(&x->tmA, in, K2, (uint64_t)rows, (uint64_t)ldo_floats * 4, BK, BM))
    return cudaErrorInvalidValue;
  if (!encode_2d(&x->tmBhi, Bhi, P, P, P * 4, BK, BN)) return cudaErrorInvalidValue;
  if (!encode_2d(&x->tmBlo, Blo, P, P, P * 4, BK, BN)) return cudaErrorInvalidValue;
  return cudaSuccess;
}

cudaError_t launch_xform_tc(const XformTc& x, int* err, cudaStream_t st) {
  const size_t smem = (size_t)STAGES * STAGE_BYTES + 1024;
  cudaError_t e =
      cudaFuncSetAttribute(k_xform_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  if (x.rows == 0) return cudaSuccess;
  dim3 grid((x.rows + BM - 1) / BM, x.nblk_n);
  k_xform_tc<<<grid, NTHREADS, smem, st>>>(x.tmA, x.tmBhi, x.tmBlo, x.out, x.rows, x.ncols, x.ldo,
                                           x.kchunks, err);
  return cudaGetLastError();
}
