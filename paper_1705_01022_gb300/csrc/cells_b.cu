// Coarse-cell device-step kernels (cells.cuh) for the cell shapes 8x16, 16x4, 16x8, 16x16.
#include "cells.cuh"

namespace oct {

template void launch_cells_shape<8, 16>(const StepArgs &, bool, const dim3 &, const dim3 &,
                                          cudaStream_t);
template void launch_cells_shape<16, 4>(const StepArgs &, bool, const dim3 &, const dim3 &,
                                          cudaStream_t);
template void launch_cells_shape<16, 8>(const StepArgs &, bool, const dim3 &, const dim3 &,
                                          cudaStream_t);
template void launch_cells_shape<16, 16>(const StepArgs &, bool, const dim3 &, const dim3 &,
                                          cudaStream_t);

}  // namespace oct
