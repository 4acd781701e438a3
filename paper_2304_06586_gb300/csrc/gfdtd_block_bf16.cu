// gfdtd_block_bf16.cu -- instantiations of the batched time-block kernel for
// __nv_bfloat16 field storage (one translation unit per precision so they compile in
// parallel).
#include "gfdtd_block.cuh"

namespace gfdtd {

#define GFDTD_SHAPES(X) X(16, 16) X(8, 16)

int block_launch_bf16(int matter, int C, int TB, const void* a, int grid, int block,
                       cudaStream_t st) {
#define X(c, tb)                                                                     \
  if (C == c && TB == tb)                                                            \
    return matter ? launch_block_shape<c, tb, true, __nv_bfloat16>(a, grid, block, st)          \
                  : launch_block_shape<c, tb, false, __nv_bfloat16>(a, grid, block, st);
  GFDTD_SHAPES(X)
#undef X
  return (int)cudaErrorInvalidValue;
}

int block_occupancy_bf16(int matter, int C, int TB, int block, int* nb) {
#define X(c, tb)                                                                     \
  if (C == c && TB == tb)                                                            \
    return matter ? occupancy_block_shape<c, tb, true, __nv_bfloat16>(block, nb)                \
                  : occupancy_block_shape<c, tb, false, __nv_bfloat16>(block, nb);
  GFDTD_SHAPES(X)
#undef X
  return (int)cudaErrorInvalidValue;
}

int block_shapes_bf16(int* C, int* TB, int max) {
  int n = 0;
#define X(c, tb) if (n < max) { C[n] = c; TB[n] = tb; ++n; }
  GFDTD_SHAPES(X)
#undef X
  return n;
}

}  // namespace gfdtd
