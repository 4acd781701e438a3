// gfdtd_block_f64.cu -- instantiations of the batched time-block kernels for
// FP64 field storage and arithmetic.  One translation unit per precision so they compile in parallel.
// A shape is (cells per lane, steps per time block, blocks per SM that the
// fast kernel's registers are limited to).
#include "gfdtd_block.cuh"

namespace gfdtd {

#define GFDTD_SHAPES(X) X(4,8,4) X(8,8,4) X(8,16,4) X(8,24,6)

int block_launch_f64(int variant, int C, int TB, int MB, const void* a, int grid, int block,
                        cudaStream_t st) {
#define X(c, tb, mb) \
  if (C == c && TB == tb && MB == mb) \
    return launch_block_shape<c, tb, double, false, mb>(variant, a, grid, block, st);
  GFDTD_SHAPES(X)
#undef X
  return (int)cudaErrorInvalidValue;
}

int block_occupancy_f64(int variant, int C, int TB, int MB, int block, int* nb) {
#define X(c, tb, mb) \
  if (C == c && TB == tb && MB == mb) return occupancy_block_shape<c, tb, double, false, mb>(variant, block, nb);
  GFDTD_SHAPES(X)
#undef X
  return (int)cudaErrorInvalidValue;
}

int block_shapes_f64(int* C, int* TB, int* MB, int max) {
  int n = 0;
#define X(c, tb, mb) if (n < max) { C[n] = c; TB[n] = tb; MB[n] = mb; ++n; }
  GFDTD_SHAPES(X)
#undef X
  return n;
}

}  // namespace gfdtd
