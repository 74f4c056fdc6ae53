// Where a warp's sub-tile lies: the device layer of one MCS (Sec. 3, DTr).
//
// The origin (ox, oy) and the set permutation come from Philox(t, 0, 0,
// MCS<<28) once per MCS; device tile (tx, ty) has index T = ty*tiles_x + tx
// (the tile index of the random streams) and its sub-tile of set sigma =
// perm[k] starts at (ox + 2Bx tx + Bx (sigma&1), oy + 2By ty + By (sigma>>1))
// mod L.  A handle may hold only a row strip of the lattice (multi-GPU strip
// partition): its buffer then starts at global row row0, and it updates the
// strip_tiles_y device-tile rows whose first row (oy + 2By ty) mod L lies in
// [row0, row0 + 2By strip_tiles_y).  Work index w counts the sub-tiles the
// launch updates; y0 is returned in buffer rows.
#pragma once
#include <cstdint>

#include "oct_internal.h"
#include "philox.cuh"
#include "subtile.cuh"

namespace oct {

struct TilePlace {
    uint32_t T;       // device-tile index (random streams)
    uint32_t x0, y0;  // sub-tile origin: global column, buffer row
};

__host__ __device__ __forceinline__ uint32_t work_tiles(const StepArgs &a) {
    return a.tiles_x * (a.strip_tiles_y ? a.strip_tiles_y : a.tiles_y);
}

__device__ __forceinline__ TilePlace place_tile(const StepArgs &a, uint32_t w, uint32_t t) {
    const uint32_t L = a.L;
    const uint4 M = philox4x32_10(t, 0u, 0u, kTagMcs << 28, a.k0, a.k1);
    const uint32_t ox = static_cast<uint32_t>((static_cast<uint64_t>(M.x) * L) >> 32);
    const uint32_t oy = static_cast<uint32_t>((static_cast<uint64_t>(M.y) * L) >> 32);
    const uint32_t pidx = static_cast<uint32_t>((static_cast<uint64_t>(M.z) * 24u) >> 32);
    const int sigma = perm_element(pidx, a.k);
    const uint32_t tx = w % a.tiles_x, j = w / a.tiles_x;
    uint32_t ty = j;
    if (a.strip_tiles_y) {
        // tile rows whose first row lies in the strip: ty = (j - q) mod tiles_y,
        // q = ((oy - row0) mod L) div 2By
        const uint32_t d = (oy + L - a.row0) % L;
        const uint32_t q = (d / (2u * a.By)) % a.tiles_y;
        ty = (j + a.tiles_y - q) % a.tiles_y;
    }
    TilePlace p;
    p.T = ty * a.tiles_x + tx;
    p.x0 = static_cast<uint32_t>(
        (static_cast<uint64_t>(ox) + 2ull * a.Bx * tx + static_cast<uint64_t>(a.Bx) * (sigma & 1)) % L);
    const uint32_t yg = static_cast<uint32_t>(
        (static_cast<uint64_t>(oy) + 2ull * a.By * ty + static_cast<uint64_t>(a.By) * (sigma >> 1)) % L);
    p.y0 = (yg + L - a.row0) % L;
    return p;
}

}  // namespace oct
