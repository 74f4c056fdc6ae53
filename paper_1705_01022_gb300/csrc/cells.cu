// Device step of DTrDT with thread cells coarser than 4x4 sites (cells.cuh):
// the shapes with a kernel and the dispatch of one device step to them.
#include "oct_internal.h"

namespace oct {

template <int CX, int CY>
void launch_cells_shape(const StepArgs &a, bool any_random, const dim3 &grid, const dim3 &block, cudaStream_t st);

bool cells_shape_supported(int cx, int cy) {
    switch (cx * 100 + cy) {
        case 804: case 408: case 808: case 1604: case 1608: case 816: case 1616:
        case 3204: case 3208: case 3216: case 416:
            return true;
        default:
            return false;
    }
}

cudaError_t launch_cells_step(const StepArgs &a, bool any_random, cudaStream_t st) {
    const uint32_t n_tiles = a.tiles_x * (a.strip_tiles_y ? a.strip_tiles_y : a.tiles_y);
    const dim3 grid((n_tiles + kStepWarpsPerBlock - 1) / kStepWarpsPerBlock), block(kStepWarpsPerBlock * 32);
    switch (a.cx * 100 + a.cy) {
        case 804: launch_cells_shape<8, 4>(a, any_random, grid, block, st); break;
        case 408: launch_cells_shape<4, 8>(a, any_random, grid, block, st); break;
        case 808: launch_cells_shape<8, 8>(a, any_random, grid, block, st); break;
        case 1604: launch_cells_shape<16, 4>(a, any_random, grid, block, st); break;
        case 1608: launch_cells_shape<16, 8>(a, any_random, grid, block, st); break;
        case 816: launch_cells_shape<8, 16>(a, any_random, grid, block, st); break;
        case 1616: launch_cells_shape<16, 16>(a, any_random, grid, block, st); break;
        case 3204: launch_cells_shape<32, 4>(a, any_random, grid, block, st); break;
        case 3208: launch_cells_shape<32, 8>(a, any_random, grid, block, st); break;
        case 3216: launch_cells_shape<32, 16>(a, any_random, grid, block, st); break;
        case 416: launch_cells_shape<4, 16>(a, any_random, grid, block, st); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace oct
