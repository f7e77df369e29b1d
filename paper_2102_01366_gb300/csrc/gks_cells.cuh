// gks_cells.cuh -- lane layout of the cell kernels, shared by the
// translation units that hold them.
#pragma once

#include <cstdint>

#include "gks_kernels.h"

namespace gks {

// 5 lanes per cell (one per conservative component), 6 cells per warp (lanes
// 30, 31 idle), CELLS_PER_BLOCK cells per 128-thread block
struct CellLane {
    int64_t c;    // cell (clamped to a valid cell on idle lanes)
    int q;        // component
    int base;     // lane of component 0 of this cell
    bool active;  // lane carries a real (cell, component)
};

__device__ __forceinline__ CellLane cell_lane(int64_t nc) {
    CellLane L;
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int cl = lane / 5;
    L.q = lane - 5 * cl;
    L.base = lane - L.q;
    const int64_t c = (int64_t)blockIdx.x * CELLS_PER_BLOCK + warp * 6 + cl;
    L.active = lane < 30 && c < nc;
    L.c = c < nc ? c : nc - 1;
    return L;
}


static inline unsigned cell_grid(int64_t nc) { return (unsigned)((nc + CELLS_PER_BLOCK - 1) / CELLS_PER_BLOCK); }

}  // namespace gks
