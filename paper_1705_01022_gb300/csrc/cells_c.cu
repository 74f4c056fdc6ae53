// Coarse-cell device-step kernels (cells.cuh) for the cell shapes 32x4, 32x8, 32x16.
#include "cells.cuh"

namespace oct {

template void launch_cells_shape<32, 4>(const StepArgs &, bool, const dim3 &, const dim3 &,
                                          cudaStream_t);
template void launch_cells_shape<32, 8>(const StepArgs &, bool, const dim3 &, const dim3 &,
                                          cudaStream_t);
template void launch_cells_shape<32, 16>(const StepArgs &, bool, const dim3 &, const dim3 &,
                                          cudaStream_t);

}  // namespace oct
