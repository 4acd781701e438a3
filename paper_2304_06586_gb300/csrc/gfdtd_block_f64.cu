// gfdtd_block_f64.cu -- instantiations of the batched time-block kernel for
// double field storage (one translation unit per precision so they compile in
// parallel).
#include "gfdtd_block.cuh"

namespace gfdtd {

#define GFDTD_SHAPES(X) X(8, 8) X(8, 16)

int block_launch_f64(int matter, int C, int TB, const void* a, int grid, int block,
                       cudaStream_t st) {
#define X(c, tb)                                                                     \
  if (C == c && TB == tb)                                                            \
    return matter ? launch_block_shape<c, tb, true, double>(a, grid, block, st)          \
                  : launch_block_shape<c, tb, false, double>(a, grid, block, st);
  GFDTD_SHAPES(X)
#undef X
  return (int)cudaErrorInvalidValue;
}

int block_occupancy_f64(int matter, int C, int TB, int block, int* nb) {
#define X(c, tb)                                                                     \
  if (C == c && TB == tb)                                                            \
    return matter ? occupancy_block_shape<c, tb, true, double>(block, nb)                \
                  : occupancy_block_shape<c, tb, false, double>(block, nb);
  GFDTD_SHAPES(X)
#undef X
  return (int)cudaErrorInvalidValue;
}

int block_shapes_f64(int* C, int* TB, int max) {
  int n = 0;
#define X(c, tb) if (n < max) { C[n] = c; TB[n] = tb; ++n; }
  GFDTD_SHAPES(X)
#undef X
  return n;
}

}  // namespace gfdtd
