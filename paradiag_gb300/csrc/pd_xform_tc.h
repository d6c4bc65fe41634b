// Host interface of the tcgen05 x-eigentransform (pd_xform_tc.cu).
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>

// Prepared launch of one direction of the transform: TMA descriptors of the
// input rows and of the split operator G = G_hi + G_lo (row-major,
// bpad x bpad floats, zero-padded), and the output geometry.
struct XformTc {
  CUtensorMap tmA, tmBhi, tmBlo;
  int rows, ncols, ldo, kchunks, nblk_n;
  float* out;
};

// padded size (multiple of 256) of the real operator for nx complex points
size_t xform_tc_bpad(int nx);
// rows: spectrum rows; ldo_floats: row stride of input and output in floats
// (2 * padded nx, a multiple of 4); in/out: device spectra; Bhi/Blo: device
// operator halves.
cudaError_t xform_tc_prepare(XformTc* x, int rows, int nx, int ldo_floats, const float* in,
                             float* out, const float* Bhi, const float* Blo);
cudaError_t launch_xform_tc(const XformTc& x, int* err, cudaStream_t st);
