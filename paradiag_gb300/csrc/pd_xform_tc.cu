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
// Precision: FP16 operands split in two terms, FP32 accumulation.  With power-
// of-two scales sA (from the largest |A|, recorded by the kernel that wrote A)
// and sG, a = sA A = a_hi + a_lo and g = sG G = g_hi + g_lo with a_hi = fp16(a),
// a_lo = fp16(a - a_hi); D = (a_hi g_hi + a_hi g_lo + a_lo g_hi) / (sA sG).
// Each term carries 11 significand bits, so values within 2^-18 of the largest
// keep about 22 bits (the dropped a_lo g_lo is ~2^-22 relative) and smaller
// ones an absolute error below 2^-40 of the largest: an FP32-level transform in
// the 2-norm, at twice the TF32 MMA rate and half the operand bytes of split
// TF32.  A is loaded by TMA as FP32 and split in place in shared memory; G is
// split on the host.
//
// Persistent kernel, one CTA per SM walking tiles of 128 x 256 (M x N); K
// chunks of 32 (one 64-byte swizzle row of FP16) through four pipeline stages
// that keep streaming across tile boundaries.  Warp roles: warp 0 issues TMA
// loads, warp 1 allocates TMEM and issues the MMAs (one elected thread) into
// one of two accumulators, warps 2-5 split A (one row per thread), warps 6-9
// drain the other accumulator (tcgen05.ld) to global memory, so the epilogue of
// a tile runs under the MMAs of the next.  The N blocks of one row block are
// consecutive tiles, so A comes from DRAM once.  Every mbarrier wait is
// bounded; on a timeout the CTA records an error bit, waits for its MMAs and
// loads in flight, frees its TMEM and returns.
#include <cuda.h>
#include <cuda_fp16.h>

#include <cmath>
#include <vector>

#include "pd_internal.h"
#include "pd_xform_tc.h"

namespace {

constexpr int BM = 128, BN = 256;
constexpr int KH = 32;                  // FP16 K elements per stage (64 bytes)
constexpr int AF_BOX = 16;              // FP32 K elements per TMA box of A (64 bytes)
constexpr int A_BYTES = BM * KH * 4;    // 16 KB: FP32 A, then A_hi | A_lo in FP16
constexpr int B_BYTES = BN * KH * 2;    // 16 KB per operand half
constexpr int STAGE_BYTES = A_BYTES + 2 * B_BYTES;
constexpr int STAGES = 4;
// unused shared memory after the last stage, so that every operand read of the
// tensor cores stays inside the CTA's allocation
constexpr int GUARD_BYTES = 32 * 1024;
constexpr int TMEM_COLS = 2 * BN;   // two accumulators: epilogue of one tile under the MMAs of the next
// XTC_UDF_ADD: a ring of EG slots per epilogue warp, each the iterate of 16
// time levels for the warp's 32 points (4 KB), filled by cp.async
constexpr int EG = 3;
constexpr int EPI_STAGE_BYTES = 4 * EG * 16 * 32 * 8;
constexpr int NTHREADS = 320;
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
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t phase, volatile int* abort_flag,
                                          long long limit) {
  for (long long i = 0; i < limit; ++i) {
    if (mbar_try(bar, phase)) return true;
    if ((i & 255) == 255 && *abort_flag) return false;
  }
  *abort_flag = 1;
  return false;
}

// bounded wait for work already issued (loads or MMAs in flight) before the
// CTA frees its resources; does not stop early on the abort flag
__device__ __forceinline__ void mbar_drain(uint32_t bar, uint32_t phase) {
  for (long long i = 0; i < WAIT_LIMIT; ++i)
    if (mbar_try(bar, phase)) return;
}

__device__ __forceinline__ void tma_load_4d(uint32_t dst, const CUtensorMap* map, int c0, int c1,
                                            int c2, int c3, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, "
      "%3, %4, %5}], [%6];" ::"r"(dst),
      "l"(map), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(bar)
      : "memory");
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, int c0, int c1,
                                            uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, "
      "%3}], [%4];" ::"r"(dst),
      "l"(map), "r"(c0), "r"(c1), "r"(bar)
      : "memory");
}

// shared-memory matrix descriptor: K-major, 64-byte swizzle, 8-row groups
// 512 bytes apart (tcgen05 descriptor format: start >> 4 in bits 0-13, leading
// offset >> 4 in 16-29, stride offset >> 4 in 32-45, version 1 in 46-47,
// swizzle mode in 61-63 with 4 = 64-byte swizzle)
__device__ __forceinline__ uint64_t sdesc(uint32_t addr) {
  uint64_t d = 0;
  d |= (uint64_t)((addr & 0x3FFFF) >> 4);
  d |= (uint64_t)1 << 16;
  d |= (uint64_t)(512 >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)4 << 61;
  return d;
}

// instruction descriptor of kind::f16: D f32 (bits 4-5 = 1), A and B f16
// (bits 7-9 and 10-12 = 0), both K-major, N >> 3 in bits 17-22, M >> 4 in 24-28
constexpr uint32_t IDESC = (1u << 4) | ((uint32_t)(BN >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);

__device__ __forceinline__ void mma_f16(uint32_t tmem, uint64_t a, uint64_t b, uint32_t acc) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(tmem),
      "l"(a), "l"(b), "r"(IDESC), "r"(acc)
      : "memory");
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
      : "memory");
}

// power-of-two scale s with s |x| < 2^15 for |x| <= amax (1 when amax is 0 or
// not finite)
__device__ __forceinline__ float a_scale(float amax) {
  if (!(amax > 0.f) || !isfinite(amax)) return 1.f;
  int e;
  frexpf(amax, &e);  // amax < 2^e
  e = max(-100, min(100, e));
  return ldexpf(1.f, 15 - e);
}

// split 8 scaled FP32 values into FP16 high and low parts (8 halves each)
__device__ __forceinline__ void split8(const float* v, float s, uint4& hi, uint4& lo) {
  uint32_t h[4], l[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const float x0 = v[2 * q] * s, x1 = v[2 * q + 1] * s;
    const __half2 hh = __floats2half2_rn(x0, x1);
    const float2 hf = __half22float2(hh);
    const __half2 ll = __floats2half2_rn(x0 - hf.x, x1 - hf.y);
    h[q] = *reinterpret_cast<const uint32_t*>(&hh);
    l[q] = *reinterpret_cast<const uint32_t*>(&ll);
  }
  hi = make_uint4(h[0], h[1], h[2], h[3]);
  lo = make_uint4(l[0], l[1], l[2], l[3]);
}

// epilogue targets of the time contractions (XformTc, modes XTC_SPEC / XTC_UDF_*)
struct XtcEpi {
  int a_blocked;    // A in 128 x 16 blocks (xform_tc_prepare_blocked), loaded by a 4D map
  int stall_chunk;  // testing aid: CTA 0 issues no loads from this chunk on (-1: none)
  long long wait_limit;   // iterations of a bounded mbarrier wait
  SpecGeom sg;
  float2* spec;
  unsigned* spec_amax;
  unsigned* spec_amax_reset;
  float2* Udf;
  int* flag;
};

template <int EPI>
__global__ void __launch_bounds__(NTHREADS, 1)
    k_xform_tc(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmBhi,
               const __grid_constant__ CUtensorMap tmBlo, float* __restrict__ out, int rows,
               int ncols, int ldo, int kchunks, int nblk_n, int ntiles,
               const unsigned* __restrict__ amax_bits, float g_inv, int* err, const XtcEpi ep) {
  // operand stages: two in the update mode, whose epilogue stages the iterate
  // in the memory the other two would take
  constexpr int NS = EPI == XTC_UDF_ADD ? 2 : STAGES;
  extern __shared__ __align__(1024) unsigned char smraw[];
  // 1024-byte aligned operand stages (the swizzle patterns repeat every 512 bytes)
  unsigned char* base = (unsigned char*)(((uintptr_t)smraw + 1023) & ~(uintptr_t)1023);
  __shared__ __align__(8) uint64_t bar_full[NS], bar_split[NS], bar_empty[NS];
  __shared__ __align__(8) uint64_t bar_accf[2], bar_acce[2], bar_done;
  __shared__ uint32_t tmem_slot;
  __shared__ int abort_flag;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const float sa = a_scale(__uint_as_float(*amax_bits));

  if (threadIdx.x == 0) {
    for (int s = 0; s < NS; ++s) {
      mbar_init(smem_u32(&bar_full[s]), 1);
      mbar_init(smem_u32(&bar_split[s]), 4);
      mbar_init(smem_u32(&bar_empty[s]), 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(smem_u32(&bar_accf[b]), 1);
      mbar_init(smem_u32(&bar_acce[b]), 4);
    }
    mbar_init(smem_u32(&bar_done), 1);
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

  // stage layout: [A: FP32 boxes 0 | 1, split in place to A_hi | A_lo] [G_hi] [G_lo]
  auto stage_ptr = [&](int s, int which) -> unsigned char* {
    const int off[4] = {0, A_BYTES / 2, A_BYTES, A_BYTES + B_BYTES};
    return base + (size_t)s * STAGE_BYTES + off[which];
  };
  // tiles of this CTA: T = blockIdx.x + i gridDim.x; T -> (row block, N block)
  // with the N blocks of one row block consecutive
  const int my_tiles = blockIdx.x < ntiles ? (ntiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;

  if (warp == 0) {
    // ---------------- TMA producer: one chunk counter g over all tiles
    if (lane == 0) {
      int g = 0;
      bool ok = true;
      for (int i = 0; i < my_tiles && ok; ++i) {
        const int T = blockIdx.x + i * gridDim.x;
        const int r0 = (T / nblk_n) * BM, n0 = (T % nblk_n) * BN;
        for (int c = 0; c < kchunks; ++c, ++g) {
          const int s = g % NS;
          const uint32_t u = (uint32_t)(g / NS);
          if (blockIdx.x == 0 && g == ep.stall_chunk) {
            // withheld: nothing of this chunk is in flight, so the consumers'
            // bounded waits run out and the CTA takes its abort path
            ok = false;
            break;
          }
          if (g >= NS && !mbar_wait(smem_u32(&bar_empty[s]), (u & 1u) ^ 1u, abortp, ep.wait_limit)) {
            ok = false;
            break;
          }
          const uint32_t fb = smem_u32(&bar_full[s]);
          mbar_expect_tx(fb, (uint32_t)(A_BYTES + 2 * B_BYTES));
          if (ep.a_blocked) {
            // blocks (k / 16, row / 128) of 128 rows x 16 floats, contiguous
            tma_load_4d(smem_u32(stage_ptr(s, 0)), &tmA, 0, 0, 2 * c, r0 / BM, fb);
            tma_load_4d(smem_u32(stage_ptr(s, 1)), &tmA, 0, 0, 2 * c + 1, r0 / BM, fb);
          } else {
            tma_load_2d(smem_u32(stage_ptr(s, 0)), &tmA, c * KH, r0, fb);
            tma_load_2d(smem_u32(stage_ptr(s, 1)), &tmA, c * KH + AF_BOX, r0, fb);
          }
          tma_load_2d(smem_u32(stage_ptr(s, 2)), &tmBhi, c * KH, n0, fb);
          tma_load_2d(smem_u32(stage_ptr(s, 3)), &tmBlo, c * KH, n0, fb);
        }
      }
      // drain: wait for the loads still in flight before the CTA may exit
      for (int q = (g > NS ? g - NS : 0); q < g; ++q)
        mbar_drain(smem_u32(&bar_full[q % NS]), (uint32_t)((q / NS) & 1));
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer: accumulator buffer i & 1 for local tile i
    if (lane == 0) {
      int g = 0;
      bool ok = true;
      for (int i = 0; i < my_tiles && ok; ++i) {
        const int ab = i & 1;
        const uint32_t v = (uint32_t)(i >> 1);
        if (i >= 2 && !mbar_wait(smem_u32(&bar_acce[ab]), (v & 1u) ^ 1u, abortp, ep.wait_limit)) {
          ok = false;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t acc = tmem + (uint32_t)(ab * BN);
        for (int c = 0; c < kchunks; ++c, ++g) {
          const int s = g % NS;
          const uint32_t u = (uint32_t)(g / NS);
          if (!mbar_wait(smem_u32(&bar_split[s]), u & 1u, abortp, ep.wait_limit)) { ok = false; break; }
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          const uint32_t ahi = smem_u32(stage_ptr(s, 0)), alo = smem_u32(stage_ptr(s, 1));
          const uint32_t bhi = smem_u32(stage_ptr(s, 2)), blo = smem_u32(stage_ptr(s, 3));
#pragma unroll
          for (int kk = 0; kk < KH / 16; ++kk) {
            const uint32_t koff = kk * 32;  // 16 halves = 32 bytes along the 64-byte row
            const uint32_t first = (c == 0 && kk == 0) ? 0u : 1u;
            mma_f16(acc, sdesc(ahi + koff), sdesc(bhi + koff), first);
            mma_f16(acc, sdesc(ahi + koff), sdesc(blo + koff), 1u);
            mma_f16(acc, sdesc(alo + koff), sdesc(bhi + koff), 1u);
          }
          mma_commit(smem_u32(&bar_empty[s]));
        }
        if (ok) mma_commit(smem_u32(&bar_accf[ab]));
      }
      // every MMA issued so far has completed once bar_done fires
      mma_commit(smem_u32(&bar_done));
      mbar_drain(smem_u32(&bar_done), 0u);
    }
  } else if (warp < 6) {
    // ---------------- A split (warps 2-5, thread t owns row t of the block)
    const int t = threadIdx.x - 64;  // 0..127
    // 64-byte swizzle of 64-byte rows: 16-byte chunk c of row t sits at
    // c ^ ((t >> 1) & 3)
    const int sw = (t >> 1) & 3;
    const int nchunks = my_tiles * kchunks;
    for (int g = 0; g < nchunks; ++g) {
      const int s = g % NS;
      const uint32_t u = (uint32_t)(g / NS);
      if (!mbar_wait(smem_u32(&bar_full[s]), u & 1u, abortp, ep.wait_limit)) break;
      unsigned char* a0 = stage_ptr(s, 0) + t * 64;  // row t of box 0 / of A_hi
      unsigned char* a1 = stage_ptr(s, 1) + t * 64;  // row t of box 1 / of A_lo
      // the whole row (32 FP32 values) into registers before it is overwritten
      float v[32];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const float4 x0 = *reinterpret_cast<const float4*>(a0 + ((q ^ sw) << 4));
        const float4 x1 = *reinterpret_cast<const float4*>(a1 + ((q ^ sw) << 4));
        v[4 * q] = x0.x; v[4 * q + 1] = x0.y; v[4 * q + 2] = x0.z; v[4 * q + 3] = x0.w;
        v[16 + 4 * q] = x1.x; v[17 + 4 * q] = x1.y; v[18 + 4 * q] = x1.z; v[19 + 4 * q] = x1.w;
      }
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        uint4 h, l;
        split8(v + 8 * q, sa, h, l);
        *reinterpret_cast<uint4*>(a0 + ((q ^ sw) << 4)) = h;
        *reinterpret_cast<uint4*>(a1 + ((q ^ sw) << 4)) = l;
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      __syncwarp();
      if (lane == 0) mbar_arrive(smem_u32(&bar_split[s]));
    }
  } else {
    // ---------------- epilogue (warps 6-9): TMEM lanes 32*(warp % 4) .. +31
    // hold rows r0 + that range of the tile
    const float oscale = g_inv / sa;  // exact: both are powers of two
    const int q4 = warp & 3;
    float amx = 0.f;                  // XTC_SPEC: max |D| over this thread's outputs
    bool bad = false;                 // XTC_UDF_*: a non-finite increment
    if constexpr (EPI == XTC_SPEC) {
      if (blockIdx.x == 0 && warp == 6 && lane == 0 && ep.spec_amax_reset) *ep.spec_amax_reset = 0u;
    }
    // XTC_UDF_ADD: the iterate of the CTA's column blocks (16 time levels of
    // one tile; block q = local tile q / 16, columns 16 (q % 16)) streams
    // through ring slot q % EG of this warp by cp.async, EG - 1 blocks ahead of
    // its update and across tile boundaries (the iterate does not depend on
    // the MMAs, and tiles cover disjoint parts of it).  Each lane copies and
    // later reads only its own point: no cross-lane synchronisation.
    constexpr int QB = BN / 16;
    float2* ring = reinterpret_cast<float2*>(base + (size_t)NS * STAGE_BYTES + GUARD_BYTES) +
                   (size_t)(warp - 6) * (EG * 16 * 32) + lane;
    auto fill = [&](int q) {
      const int ti = q / QB, jb = q % QB;
      if (ti < my_tiles) {
        const int Tq = blockIdx.x + ti * gridDim.x;
        const int rq = (Tq / nblk_n) * BM + q4 * 32 + lane, nq = (Tq % nblk_n) * BN + jb * 16;
        if (rq < rows) {
          float2* d = ring + (q % EG) * (16 * 32);
#pragma unroll
          for (int u = 0; u < 16; ++u)
            if (nq + u < ncols)
              asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(smem_u32(d + u * 32)),
                           "l"(ep.Udf + (size_t)(nq + u) * rows + rq)
                           : "memory");
        }
      }
      asm volatile("cp.async.commit_group;" ::: "memory");
    };
    if constexpr (EPI == XTC_UDF_ADD) {
      for (int q = 0; q < EG - 1; ++q) fill(q);
    }
    for (int i = 0; i < my_tiles; ++i) {
      const int ab = i & 1;
      const uint32_t v2 = (uint32_t)(i >> 1);
      if (!mbar_wait(smem_u32(&bar_accf[ab]), v2 & 1u, abortp, ep.wait_limit)) break;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const int T = blockIdx.x + i * gridDim.x;
      const int r0 = (T / nblk_n) * BM, n0 = (T % nblk_n) * BN;
      const int row = r0 + q4 * 32 + lane;
      for (int j = 0; j < BN; j += 16) {
        const int qc = i * QB + j / 16;     // this column block's place in the stream
        if constexpr (EPI == XTC_UDF_ADD) {
          fill(qc + EG - 1);
          // the groups of blocks up to qc are complete
          asm volatile("cp.async.wait_group %0;" ::"n"(EG - 1) : "memory");
        }
        uint32_t v[16];
        const uint32_t taddr = tmem + ((uint32_t)(q4 * 32) << 16) + (uint32_t)(ab * BN + j);
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,"
            "%13,%14,%15}, [%16];"
            : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
              "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]),
              "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
            : "r"(taddr));
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        const int n = n0 + j;
        if (row >= rows) continue;
        if constexpr (EPI == XTC_ROWS) {
          float* o = out + (size_t)row * ldo + n;
          if (n + 16 <= ncols) {
#pragma unroll
            for (int u = 0; u < 4; ++u)
              reinterpret_cast<float4*>(o)[u] = make_float4(
                  __uint_as_float(v[4 * u]) * oscale, __uint_as_float(v[4 * u + 1]) * oscale,
                  __uint_as_float(v[4 * u + 2]) * oscale, __uint_as_float(v[4 * u + 3]) * oscale);
          } else {
#pragma unroll
            for (int u = 0; u < 16; ++u)
              if (n + u < ncols) o[u] = __uint_as_float(v[u]) * oscale;
          }
        } else if constexpr (EPI == XTC_SPEC) {
          // row = spatial point s; columns n, n + 1 = (re, im) of spectrum row n / 2
          // (n even): the lanes of a warp write consecutive points of one row
          const size_t off = spec_index(ep.sg, 0, row);
#pragma unroll
          for (int u = 0; u < 8; ++u) {
            if (n + 2 * u >= ncols) break;
            const float re = __uint_as_float(v[2 * u]) * oscale;
            const float im = __uint_as_float(v[2 * u + 1]) * oscale;
            ep.spec[(size_t)((n >> 1) + u) * ep.sg.specS + off] = make_float2(re, im);
            amx = fmaxf(amx, fmaxf(fabsf(re), fabsf(im)));
          }
        } else {
          // row = spatial point s, column = time level: Udf[(n + u) rows + s]
#pragma unroll
          for (int u = 0; u < 16; ++u) {
            if (n + u >= ncols) break;
            const float d = __uint_as_float(v[u]) * oscale;
            bad |= !isfinite(d);
            float2* up = ep.Udf + (size_t)(n + u) * rows + row;
            if constexpr (EPI == XTC_UDF_SET) {
              *up = make_float2(d, 0.f);
            } else {
              const float2 uo = ring[(qc % EG) * (16 * 32) + u * 32];
              df t = two_sum(uo.x, d);
              t = fast_two_sum(t.hi, t.lo + uo.y);
              *up = make_float2(t.hi, t.lo);
            }
          }
        }
      }

      // this warp's reads of accumulator ab are complete: hand it back
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncwarp();
      if (lane == 0) mbar_arrive(smem_u32(&bar_acce[ab]));
    }
    // copies still in flight (blocks past the last tile are empty groups; after
    // an abort, blocks of tiles not reached) finish before the CTA exits
    if constexpr (EPI == XTC_UDF_ADD) asm volatile("cp.async.wait_group 0;" ::: "memory");
    if constexpr (EPI == XTC_SPEC) {
      for (int o = 16; o > 0; o >>= 1) amx = fmaxf(amx, __shfl_xor_sync(0xffffffffu, amx, o));
      if (lane == 0 && ep.spec_amax) atomicMax(ep.spec_amax, __float_as_uint(amx));
    } else if constexpr (EPI == XTC_UDF_SET || EPI == XTC_UDF_ADD) {
      if (__any_sync(0xffffffffu, bad) && lane == 0 && ep.flag) atomicOr(ep.flag, 1);
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

bool encode_2d(CUtensorMap* m, CUtensorMapDataType dt, const void* ptr, uint64_t inner,
               uint64_t outer, uint64_t row_bytes, uint32_t box_inner, uint32_t box_outer) {
  EncodeTiledFn fn = encode_fn();
  if (!fn) return false;
  const cuuint64_t dims[2] = {inner, outer};
  const cuuint64_t strides[1] = {row_bytes};
  const cuuint32_t box[2] = {box_inner, box_outer};
  const cuuint32_t estr[2] = {1, 1};
  return fn(m, dt, 2, const_cast<void*>(ptr), dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B,
            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace

size_t xform_tc_bpad(int nx) { return (size_t)(((2 * nx + BN - 1) / BN) * BN); }

float xform_tc_split(const std::vector<float>& G, std::vector<uint16_t>& hi,
                     std::vector<uint16_t>& lo) {
  float gmax = 0.f;
  for (float g : G) gmax = std::max(gmax, std::fabs(g));
  int e = 0;
  if (gmax > 0.f) std::frexp(gmax, &e);
  const float sg = std::ldexp(1.f, 14 - e);  // sg |G| < 2^14
  hi.assign(G.size(), 0);
  lo.assign(G.size(), 0);
  for (size_t i = 0; i < G.size(); ++i) {
    const float g = G[i] * sg;
    const __half h = __float2half_rn(g);
    const __half l = __float2half_rn(g - __half2float(h));
    memcpy(&hi[i], &h, 2);
    memcpy(&lo[i], &l, 2);
  }
  return 1.f / sg;
}

cudaError_t xform_tc_prepare(XformTc* x, int rows, int nx, int ldo_floats, const float* in,
                             float* out, const void* Ghi, const void* Glo, float g_inv,
                             const unsigned* amax) {
  const uint64_t K2 = 2 * (uint64_t)nx;
  const uint64_t P = xform_tc_bpad(nx);
  x->rows = rows;
  x->ncols = (int)K2;
  x->ldo = ldo_floats;
  x->kchunks = (int)((K2 + KH - 1) / KH);
  x->nblk_n = (int)(P / BN);
  x->out = out;
  x->amax = amax;
  x->g_inv = g_inv;
  if ((ldo_floats * 4) % 16 != 0) return cudaErrorInvalidValue;
  if (!encode_2d(&x->tmA, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, in, K2, (uint64_t)rows,
                 (uint64_t)ldo_floats * 4, AF_BOX, BM))
    return cudaErrorInvalidValue;
  if (!encode_2d(&x->tmBhi, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, Ghi, P, P, P * 2, KH, BN))
    return cudaErrorInvalidValue;
  if (!encode_2d(&x->tmBlo, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, Glo, P, P, P * 2, KH, BN))
    return cudaErrorInvalidValue;
  return cudaSuccess;
}

template <int EPI>
cudaError_t launch_epi(const XformTc& x, int* err, cudaStream_t st, int grid, int ntiles) {
  const size_t smem = EPI == XTC_UDF_ADD
                          ? (size_t)2 * STAGE_BYTES + 1024 + GUARD_BYTES + EPI_STAGE_BYTES
                          : (size_t)STAGES * STAGE_BYTES + 1024 + GUARD_BYTES;
  cudaError_t e =
      cudaFuncSetAttribute(k_xform_tc<EPI>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  if (grid == 0) return cudaSuccess;
  XtcEpi ep;
  ep.a_blocked = x.a_blocked;
  ep.stall_chunk = x.stall_chunk;
  ep.wait_limit = x.stall_chunk >= 0 ? (1LL << 16) : WAIT_LIMIT;
  ep.sg.specS = x.specS;
  ep.sg.nx = x.sx_nx;
  ep.sg.nxp = x.sx_nxp;
  ep.spec = x.spec;
  ep.spec_amax = x.spec_amax;
  ep.spec_amax_reset = x.spec_amax_reset;
  ep.Udf = x.Udf;
  ep.flag = x.flag;
  k_xform_tc<EPI><<<grid, NTHREADS, smem, st>>>(x.tmA, x.tmBhi, x.tmBlo, x.out, x.rows, x.ncols,
                                                x.ldo, x.kchunks, x.nblk_n, ntiles, x.amax,
                                                x.g_inv, err, ep);
  return cudaGetLastError();
}

cudaError_t xform_tc_prepare_blocked(XformTc* x, int rows, int K, const float* in,
                                     const void* Ghi, const void* Glo, float g_inv,
                                     const unsigned* amax) {
  if (K % 16 != 0 || K < 32) return cudaErrorInvalidValue;
  cudaError_t e = xform_tc_prepare(x, rows, K / 2, K, in, nullptr, Ghi, Glo, g_inv, amax);
  if (e != cudaSuccess) return e;
  EncodeTiledFn fn = encode_fn();
  if (!fn) return cudaErrorInvalidValue;
  const uint64_t rblk = (uint64_t)(rows + BM - 1) / BM;
  const cuuint64_t dims[4] = {16, (cuuint64_t)BM, (cuuint64_t)(K / 16), rblk};
  const cuuint64_t strides[3] = {16 * 4, (cuuint64_t)BM * 16 * 4, (cuuint64_t)(K / 16) * BM * 16 * 4};
  const cuuint32_t box[4] = {16, (cuuint32_t)BM, 1, 1};
  const cuuint32_t estr[4] = {1, 1, 1, 1};
  if (fn(&x->tmA, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, const_cast<float*>(in), dims, strides, box,
         estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B,
         CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
    return cudaErrorInvalidValue;
  x->a_blocked = 1;
  return cudaSuccess;
}

cudaError_t launch_xform_tc(const XformTc& x, int* err, cudaStream_t st) {
  // persistent: one CTA per SM over all tiles
  static int nsm = 0;
  if (nsm == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (nsm <= 0) nsm = 1;
  }
  const int ntiles = x.nblk_n * ((x.rows + BM - 1) / BM);
  const int grid = ntiles < nsm ? ntiles : nsm;
  switch (x.epi) {
    case XTC_ROWS: return launch_epi<XTC_ROWS>(x, err, st, grid, ntiles);
    case XTC_SPEC: return launch_epi<XTC_SPEC>(x, err, st, grid, ntiles);
    case XTC_UDF_SET: return launch_epi<XTC_UDF_SET>(x, err, st, grid, ntiles);
    case XTC_UDF_ADD: return launch_epi<XTC_UDF_ADD>(x, err, st, grid, ntiles);
    default: return cudaErrorInvalidValue;
  }
}
