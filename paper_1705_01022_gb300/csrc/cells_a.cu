// Coarse-cell device-step kernels (cells.cuh) for the cell shapes 4x8, 4x16, 8x4, 8x8.
#include "cells.cuh"

namespace oct {

template void launch_cells_shape<4, 8>(const StepArgs &, bool, const dim3 &, const dim3 &,
                                          cudaStream_t);
template void launch_cells_shape<4, 16>(const StepArgs &, bool, const dim3 &, const dim3 &,
                                          cudaStream_t);
template void launch_cells_shape<8, 4>(const StepArgs &, bool, const dim3 &, const dim3 &,
                                          cudaStream_t);
template void launch_cells_shape<8, 8>(const StepArgs &, bool, const dim3 &, const dim3 &,
                                          cudaStream_t);

}  // namespace oct
