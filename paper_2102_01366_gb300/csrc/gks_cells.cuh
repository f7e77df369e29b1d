// gks_cells.cuh -- lane layout of the cell kernels, shared by the
// translation units that hold them.
#pragma once

#include <cstdint>

#include "gks_kernels.h"

namespace gks {

// a barrier of `count` threads on named barrier `id` (0: the whole block)
__device__ __forceinline__ void group_barrier(int id, int count) {
    if (id == 0)
        __syncthreads();
    else
        asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(count) : "memory");
}

// A group of CELL_THREADS threads on one block of cells: the block index
// vb, the thread's index tid in the group, the group's barrier (named id,
// 0 the whole thread block) and its slice of shared memory for the block
// reductions.
struct CellGroup {
    int64_t vb;
    int tid;
    int bar_id;
    double* sv;   // [CELLS_PER_BLOCK]
    int32_t* sc;  // [CELLS_PER_BLOCK]
    double* red;  // [CELL_THREADS / 32][6]
    __device__ __forceinline__ void sync() const { group_barrier(bar_id, CELL_THREADS); }
};

// 5 lanes per cell (one per conservative component), 6 cells per warp (lanes
// 30, 31 idle), CELLS_PER_BLOCK cells per 128-thread block
struct CellLane {
    int64_t c;    // cell (clamped to a valid cell on idle lanes)
    int q;        // component
    int base;     // lane of component 0 of this cell
    bool active;  // lane carries a real (cell, component)
};

// vb: the block of CELLS_PER_BLOCK cells, tid: the thread within its
// CELL_THREADS (defaults: the launch's own block and thread)
__device__ __forceinline__ CellLane cell_lane(int64_t nc, int64_t vb, int tid) {
    CellLane L;
    const int lane = tid & 31;
    const int warp = tid >> 5;
    const int cl = lane / 5;
    L.q = lane - 5 * cl;
    L.base = lane - L.q;
    const int64_t c = vb * CELLS_PER_BLOCK + warp * 6 + cl;
    L.active = lane < 30 && c < nc;
    L.c = c < nc ? c : nc - 1;
    return L;
}

__device__ __forceinline__ CellLane cell_lane(int64_t nc) { return cell_lane(nc, blockIdx.x, threadIdx.x); }


static inline unsigned cell_grid(int64_t nc) { return (unsigned)((nc + CELLS_PER_BLOCK - 1) / CELLS_PER_BLOCK); }

}  // namespace gks
