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
};

// padded size (multiple of 256) of the real operator for nx complex points
size_t xform_tc_bpad(int nx);
// FP16 two-term split of the real operator G (bpad x bpad); returns g_inv, the
// power of two with G = (hi + lo) * g_inv
float xform_tc_split(const std::vector<float>& G, std::vector<uint16_t>& hi,
                     std::vector<uint16_t>& lo);
// rows: spectrum rows; ldo_floats: row stride of input and output in floats
// (2 * padded nx, a multiple of 4); in/out: device spectra; Ghi/Glo: device
// operator halves (FP16); amax: device word with max |in|.
cudaError_t xform_tc_prepare(XformTc* x, int rows, int nx, int ldo_floats, const float* in,
                             float* out, const void* Ghi, const void* Glo, float g_inv,
                             const unsigned* amax);
cudaError_t launch_xform_tc(const XformTc& x, int* err, cudaStream_t st);
