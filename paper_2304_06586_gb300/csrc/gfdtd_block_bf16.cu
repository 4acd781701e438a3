// gfdtd_block_bf16.cu -- instantiations of the batched time-block kernels for
// BF16 field storage (FP32 arithmetic).  One translation unit per precision so they compile in parallel.
// A shape is (cells per lane, steps per time block, blocks per SM that the
// fast kernel's registers are limited to).
#include "gfdtd_block.cuh"

namespace gfdtd {

#define GFDTD_SHAPES(X) X(16,16,4) X(8,16,4) X(16,24,8) X(24,24,6)

int block_launch_bf16(int variant, int C, int TB, int MB, const void* a, int grid, int block,
                        cudaStream_t st) {
#define X(c, tb, mb) \
  if (C == c && TB == tb && MB == mb) \
    return launch_block_shape<c, tb, __nv_bfloat16, false, mb>(variant, a, grid, block, st);
  GFDTD_SHAPES(X)
#undef X
  return (int)cudaErrorInvalidValue;
}

int block_occupancy_bf16(int variant, int C, int TB, int MB, int block, int* nb) {
#define X(c, tb, mb) \
  if (C == c && TB == tb && MB == mb) return occupancy_block_shape<c, tb, __nv_bfloat16, false, mb>(variant, block, nb);
  GFDTD_SHAPES(X)
#undef X
  return (int)cudaErrorInvalidValue;
}

int block_shapes_bf16(int* C, int* TB, int* MB, int max) {
  int n = 0;
#define X(c, tb, mb) if (n < max) { C[n] = c; TB[n] = tb; MB[n] = mb; ++n; }
  GFDTD_SHAPES(X)
#undef X
  return n;
}

}  // namespace gfdtd
