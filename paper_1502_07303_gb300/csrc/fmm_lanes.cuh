// fmm_lanes.cuh -- the layout of one 8^3 brick on the 32 lanes of a warp,
// shared by the forward march and the adjoint.
//
// Brick cell c = x + 8 y + 64 z; lane l owns the cells l + 32 k, k = 0..15,
// so x = l mod 8, y = (l / 8) mod 4 + 4 (k mod 2), z = k / 2, and every set
// of cells is a 16-bit mask per lane.  The shared-memory tile holds the brick
// with one halo layer per side (10^3, x fastest).
#pragma once

#include "fmm_internal.h"

namespace fmmgb {

// tile index of brick cell c
__device__ __forceinline__ int tile_of(int c)
{
    return 111 + (c & 7) + kTile * ((c >> 3) & 7) + kTile * kTile * (c >> 6);
}

// tile index of the cell k (0..15) of the lane with x = lx, (l / 8) mod 4 = lr
__device__ __forceinline__ int tb_of(int lx, int lr, int k)
{
    return 111 + lx + kTile * (lr + 4 * (k & 1)) + kTile * kTile * (k >> 1);
}

// Cells of this lane next (one step along x, y or z) to a cell of the set A
// (16-bit lane masks; x and y neighbours live on other lanes).
__device__ __forceinline__ unsigned neighbour_mask(unsigned A, int lane)
{
    constexpr unsigned kAll = 0xffffffffu;
    const int x = lane & 7, r = (lane >> 3) & 3;
    const unsigned axm = __shfl_up_sync(kAll, A, 1);
    const unsigned axp = __shfl_down_sync(kAll, A, 1);
    const unsigned aym = __shfl_up_sync(kAll, A, 8);
    const unsigned ayp = __shfl_down_sync(kAll, A, 8);
    const unsigned ay3 = __shfl_down_sync(kAll, A, 24);   // lanes 0..7 read row 3
    const unsigned ay0 = __shfl_up_sync(kAll, A, 24);     // lanes 24..31 read row 0
    unsigned n = (A << 2) | (A >> 2);                     // z -/+ 1
    if (x > 0)
        n |= axm;
    if (x < 7)
        n |= axp;
    if (r > 0)
        n |= aym;
    if (r < 3)
        n |= ayp;
    if (r == 0)
        n |= (ay3 << 1) & 0xAAAAu;     // y = 3 (slot k-1) -> y = 4 (odd slot k)
    if (r == 3)
        n |= (ay0 >> 1) & 0x5555u;     // y = 4 (slot k+1) -> y = 3 (even slot k)
    return n & 0xFFFFu;
}

}  // namespace fmmgb
