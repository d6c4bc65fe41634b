// Host interface of the tcgen05 x-eigentransform (pd_xform_tc.cu).
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <vector>

// Prepared launch of one direction of the transform: TMA descriptors of the
// input rows (FP32) and of the split operator G = (G_hi + G_lo) * g_inv (FP16,
// row-major bpad x bpad, zero-padded), the output geometry and the device word
// holding max |input| (float bits, written by the kernel that produced the
// input).
struct XformTc {
  CUtensorMap tmA, tmBhi, tmBlo;
  int rows, ncols, ldo, kchunks, nblk_n;
  float* out;
  const unsigned* amax;
  float g_inv;
  // epilogue: XTC_ROWS stores D row by row (out, ldo); the time contractions
  // of the hybrid ParaDiag-I path read D[s][n] with s a spatial point:
  //   XTC_SPEC:    n = 2k + c is component c of spectrum row k, stored as
  //                spec[k specS + off(s)] (complex FP32), max |D| into spec_amax
  //                and *spec_amax_reset = 0;
  //   XTC_UDF_SET / XTC_UDF_ADD: n is the time level; the double-float iterate
  //                Udf[n S + s] is set to / incremented by D (non-finite: bit 0
  //                of *flag).
  int epi = 0;
  int a_blocked = 0;      // A in blocks (xform_tc_prepare_blocked)
  // testing aid: CTA 0 withholds the loads of this chunk (its g-th K chunk)
  // and all later ones, with bounded waits of 2^16 polls, so that its
  // consumers time out and the launch reports bit 1 in *err (-1: off)
  int stall_chunk = -1;
  int specS = 0, sx_nx = 1, sx_nxp = 1;
  float2* spec = nullptr;
  unsigned* spec_amax = nullptr;
  unsigned* spec_amax_reset = nullptr;
  float2* Udf = nullptr;
  int* flag = nullptr;
};
enum { XTC_ROWS = 0, XTC_SPEC = 1, XTC_UDF_SET = 2, XTC_UDF_ADD = 3 };

// padded size (multiple of 256) of the real operator for nx complex points
size_t xform_tc_bpad(int nx);
// FP16 two-term split of the real operator G (bpad x bpad); returns g_inv, the
// power of two with G = (hi + lo) * g_inv
float xform_tc_split(const std::vector<float>& G, std::vector<uint16_t>& hi,
                     std::vector<uint16_t>& lo);
// rows: spectrum rows (or spatial points of a time contraction, with nx = K / 2
// for K = N = Nt); ldo_floats: row stride of input and output in floats
// (2 * padded nx, a multiple of 4); in/out: device spectra; Ghi/Glo: device
// operator halves (FP16); amax: device word with max |in|.
cudaError_t xform_tc_prepare(XformTc* x, int rows, int nx, int ldo_floats, const float* in,
                             float* out, const void* Ghi, const void* Glo, float g_inv,
                             const unsigned* amax);
// The time contractions of the hybrid ParaDiag-I path: D[s][n] = sum_k A[s][k]
// G[n][k] with K = N (K a multiple of 16, at least 32) and A stored in blocks:
// element (s, k) at ((s / 128) (K / 16) + k / 16) 2048 + (s % 128) 16 + k % 16
// (rounded up to whole 128-row blocks), so that every TMA box of A is one
// contiguous 8 KB block and its producer writes whole blocks.
cudaError_t xform_tc_prepare_blocked(XformTc* x, int rows, int K, const float* in,
                                     const void* Ghi, const void* Glo, float g_inv,
                                     const unsigned* amax);
cudaError_t launch_xform_tc(const XformTc& x, int* err, cudaStream_t st);
