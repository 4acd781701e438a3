// gfdtd_block_f32.cu -- instantiations of the batched time-block kernels for
// FP32 field storage with up to 16 cells per lane (gfdtd_block_f32w.cu has the
// wider shapes).  One or two translation units per precision so they compile in parallel.
// A shape is (cells per lane, steps per time block, blocks per SM that the
// fast kernel's registers are limited to).
#include "gfdtd_block.cuh"

namespace gfdtd {

#define GFDTD_SHAPES(X) X(8,16,4) X(16,16,4) X(16,24,8)

int block_launch_f32(int variant, int C, int TB, int MB, const void* a, int grid, int block,
                        cudaStream_t st) {
#define X(c, tb, mb) \
  if (C == c && TB == tb && MB == mb) \
    return launch_block_shape<c, tb, float, false, mb>(variant, a, grid, block, st);
  GFDTD_SHAPES(X)
#undef X
  return (int)cudaErrorInvalidValue;
}

int block_occupancy_f32(int variant, int C, int TB, int MB, int block, int* nb) {
#define X(c, tb, mb) \
  if (C == c && TB == tb && MB == mb) return occupancy_block_shape<c, tb, float, false, mb>(variant, block, nb);
  GFDTD_SHAPES(X)
#undef X
  return (int)cudaErrorInvalidValue;
}

int block_shapes_f32(int* C, int* TB, int* MB, int max) {
  int n = 0;
#define X(c, tb, mb) if (n < max) { C[n] = c; TB[n] = tb; MB[n] = mb; ++n; }
  GFDTD_SHAPES(X)
#undef X
  return n;
}

}  // namespace gfdtd
