// Banded axis pass: arguments and entry points shared by the CUDA-core kernels
// (fot_band.cu) and the tensor-core kernel (fot_tc.cu).
#pragma once

#include "fot_common.cuh"

namespace fot {

struct BandArgs {
  const float* x;      // [n_rows][len] input
  const float* cmax;   // [n_rows][n_chunks] chunk maxima of x * x_scale (log2 units)
  const float* lmarg;  // potential-update mode: natural log marginal, layout of y
  float* y;            // [len][n_rows] output (transposed)
  float* logsum;       // potential-update mode: optional natural-log LSE, layout of y
  int* err;
  unsigned long long* terms;   // += (row, output, m) triples evaluated on the CUDA cores
  float x_scale, c, eps;
  int n_rows, len, n_chunks, n_tiles;
};

// chunk maxima of a.x, then the per-(row, 32-output tile) plan: alpha (float), window start
// and window length (int), each n_rows * n_tiles words, consecutive in `plan`
void band_prepare(fot_ctx* c, const BandArgs& a, float* plan);

// the CUDA-core window sums for every (8-row group, tile) item; items whose 128-row block
// and tile are marked in `skip` (index (row / 128) * n_tiles + tile) are left alone
template <int MODE>
void band_simt(fot_ctx* c, const BandArgs& a, const float* plan, const unsigned char* skip);

}  // namespace fot
