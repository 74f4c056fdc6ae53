// Device step of DTrDT: one launch updates every sub-tile of one set.
//
// Method (arXiv:1705.01022):
//   * device layer, DTr (Sec. 3, Fig. 2): the lattice is cut into device
//     tiles of 2Bx x 2By sites anchored at a random origin drawn once per MCS;
//     each tile has four quadrants (sets) updated in a random order, one set
//     per device step, all sub-tiles of the set concurrently;
//   * block layer, single-hit DT (Sec. 3.1): inside a sub-tile, thread cells
//     (TC) of 4x4 sites are cut into four 2x2 sub-cells; per collective step
//     the block draws one sub-cell set d and every TC makes exactly one attempt
//     at a random site of its sub-cell d; 16 collective steps sweep the
//     sub-tile once;
//   * one attempt (Eq. (1)): a local minimum [X(s),X(s+x);Y(s),Y(s+y)] =
//     [0 1;0 1] flips to [1 0;1 0] with probability p, a local maximum the
//     other way with probability q.
//
// GB300 mapping.  One warp owns one sub-tile (or, for sub-tiles of fewer than
// 32 groups, several) for the whole device step; no block-wide barrier is
// needed.  Lane (gx, gy) holds a group of 32 x 16 sites
// (8 TCs across, 4 TC rows) as 16 X-row and 16 Y-row words in registers, so
// a collective step is a handful of 32-bit logic operations per TC row:
// selection masks from the site draw, the four-bit minimum/maximum pattern,
// and XOR flips.  The neighbour bits the update rule needs at the group edge
// (the X column just right of the group, the Y row just below it) are kept
// as copies (E, D) and refreshed by warp shuffles after every step.  Acceptance
// draws for 0 < p, q < 1 compare all 32 TCs of a lane against P32 at once on
// four random bit levels; the rare ties finish from a tail stream shared by the
// sub-tile through a ring in shared memory.
//
// Random streams (Philox-4x32-10, key = seed):
//   MCS draw  (t, 0, 0, MCS<<28): ox, oy, set permutation
//   set draw  (t, k, T, SET<<28): 2 bits per collective step
//   site draw (t, k|(s/2)<<2, T, SITE<<28|g): word m = TC row, bits 4j+2(s&1)
//             (x offset) and 4j+2(s&1)+1 (y offset) for the TC in column j
//   acceptance: bits 31..28 of the uniform of TC (j, m) are bit 4j+m of the
//             four words of (t, k|(s*8)<<2, T, ACC<<28|g); bits 27..0, needed
//             only when those tie with P32's, are the top of the next word of
//             the sub-tile's tail stream (t, k|(i/4)<<2, T, TAIL<<28)
#include "oct_internal.h"

#include "subtile.cuh"
#include "tiles.cuh"

namespace oct {
namespace {

// Lanes per sub-tile: its group count rounded up to a power of two.
__host__ __device__ inline uint32_t segment_lanes(uint32_t groups) {
    uint32_t s = 1u;
    while (s < groups) s <<= 1;
    return s;
}

// One device step.  A warp holds 32 / S sub-tiles of the set (S = segment_lanes
// of the sub-tile's G groups; PACKED when S < 32): lane l works on group l % S
// of sub-tile (warp index) * (32 / S) + l / S.  Packed sub-tiles draw their own
// sets, so the step takes the per-lane row-offset path.
// Resident blocks per SM that the register budget of a variant is sized for.
// The variants with the most live state (packed warps, DB with delayed borders
// and DTrDTr with acceptance draws) spill at the 96 registers of five blocks;
// at four blocks they do not, and run 3-4 % faster despite the lower occupancy.
constexpr int step_min_blocks(int scheme, bool packed) {
    return (packed || scheme == 2 || scheme == 3 || scheme == 7) ? kStepBlocksPerSMPacked : kStepBlocksPerSM;
}

template <bool RANDOM, int SCHEME, bool PACKED>
__global__ void __launch_bounds__(kStepWarpsPerBlock * 32, step_min_blocks(SCHEME, PACKED))
    dtrdt_step_kernel(const StepArgs a) {
    __shared__ __align__(16) uint32_t ring[kStepWarpsPerBlock * 32 * kRingWordsPerLane];
    const int lane = threadIdx.x & 31;
    const uint32_t G = a.GX * a.GY;
    const uint32_t S = PACKED ? segment_lanes(G) : 32u;
    const uint32_t per_warp = 32u / S;
    const uint32_t warp_id = blockIdx.x * kStepWarpsPerBlock + (threadIdx.x >> 5);
    const uint32_t n_tiles = work_tiles(a);
    if (warp_id * per_warp >= n_tiles) return;  // the whole warp leaves together
    const uint32_t seg = static_cast<uint32_t>(lane) / S, sub = static_cast<uint32_t>(lane) % S;
    const uint32_t w = warp_id * per_warp + seg;  // work index of the lane's sub-tile

    const uint32_t t = *a.t_ptr;
    const uint32_t L = a.L;
    // Device layer: origin and set order of this MCS (same for every warp).
    const TilePlace pl = place_tile(a, w < n_tiles ? w : 0u, t);
    const uint32_t T = pl.T, x0 = pl.x0, y0 = pl.y0;

    LaneCtx c;
    c.GX = static_cast<int>(a.GX);
    c.GY = static_cast<int>(a.GY);
    c.gx = static_cast<int>(sub) % c.GX;
    c.gy = static_cast<int>(sub) / c.GX;
    const bool active = sub < G && w < n_tiles;
    c.active = active;
    c.last = static_cast<int>(seg * S + G - 1u);
    c.t = t;
    c.k = a.k;
    c.T = T;
    c.g = sub;
    c.k0 = a.k0;
    c.k1 = a.k1;
    c.thr_p = a.thr_p;
    c.thr_q = a.thr_q;
    c.p_always = a.p_always;
    c.q_always = a.q_always;
    c.p_random = a.p_random;
    c.q_random = a.q_random;

    const uint32_t wpr = a.wpr;
    int net = 0, draws = 0, tails = 0;
    run_subtile<RANDOM, PACKED, SCHEME>(a.lat, L, a.plane_rows, wpr, a.Bx, a.By, x0, y0, active, c,
                                        ring + ((threadIdx.x >> 5) * 32 + seg * S) * kRingWordsPerLane,
                                        net, draws, tails);

    // Net flips (and acceptance draws): one atomic per warp into a spread of counters.
    const uint32_t T0 = warp_id * per_warp;  // (work index: only spreads the atomics)
    const int total = __reduce_add_sync(kFull, net);
    if (lane == 0 && total != 0)
        atomicAdd(&a.net[T0 % kNetSlots], static_cast<unsigned long long>(static_cast<long long>(total)));
    if (RANDOM) {
        const unsigned nd = __reduce_add_sync(kFull, static_cast<unsigned>(draws));
        if (lane == 0 && nd != 0u) atomicAdd(&a.draws[T0 % kNetSlots], static_cast<unsigned long long>(nd));
        // tail-stream Philox blocks stored by the lanes of the warp's sub-tiles
        const unsigned nb = __reduce_add_sync(kFull, active ? static_cast<unsigned>(tails) : 0u);
        if (lane == 0 && nb != 0u) atomicAdd(&a.tails[T0 % kNetSlots], static_cast<unsigned long long>(nb));
    }
}

__global__ void advance_t_kernel(uint32_t *t_ptr) { *t_ptr += 1u; }

}  // namespace

cudaError_t launch_dtrdt_step(const StepArgs &a, bool any_random, cudaStream_t st) {
    if (a.cx != 4u || a.cy != 4u) return launch_cells_step(a, any_random, st);
    const uint32_t n_tiles = work_tiles(a);
    // DTrDTr routes cells between the lanes of one sub-tile with warp-wide
    // shuffles whose pattern depends on its own draws: one sub-tile per warp.
    const uint32_t S = segment_lanes(a.GX * a.GY);
    const bool packed = S < 32u && a.scheme != 3u;
    const uint32_t per_block = kStepWarpsPerBlock * (packed ? 32u / S : 1u);
    const uint32_t blocks = (n_tiles + per_block - 1) / per_block;
    const dim3 grid(blocks), block(kStepWarpsPerBlock * 32);
#define OCT_LAUNCH(SCHEME, PACKED)                                                   \
    do {                                                                             \
        if (any_random)                                                              \
            dtrdt_step_kernel<true, SCHEME, PACKED><<<grid, block, 0, st>>>(a);      \
        else                                                                         \
            dtrdt_step_kernel<false, SCHEME, PACKED><<<grid, block, 0, st>>>(a);     \
    } while (0)
    switch (a.scheme) {
        case 1:
            if (packed)
                OCT_LAUNCH(1, true);
            else if (!any_random && a.p_always == 0xFFFFFFFFu && a.q_always == 0u)
                dtrdt_step_kernel<false, 6, false><<<grid, block, 0, st>>>(a);  // deposition only
            else
                OCT_LAUNCH(1, false);
            break;
        case 2:
            if (packed)
                OCT_LAUNCH(2, true);
            else if (a.p_random && a.q_random)
                dtrdt_step_kernel<true, 7, false><<<grid, block, 0, st>>>(a);  // both rates random
            else
                OCT_LAUNCH(2, false);
            break;
        case 3:
            OCT_LAUNCH(3, false);
            break;
        default:
            if (!any_random && a.p_always == 0xFFFFFFFFu && a.q_always == 0u) {
                // deposition only (the KPZ case p = 1, q = 0): no acceptance masks
                if (packed)
                    dtrdt_step_kernel<false, 4, true><<<grid, block, 0, st>>>(a);
                else
                    dtrdt_step_kernel<false, 4, false><<<grid, block, 0, st>>>(a);
            } else if (any_random && a.p_random && a.q_random) {
                // both rates strictly inside (0, 1): every candidate is decided by its draw
                if (packed)
                    dtrdt_step_kernel<true, 5, true><<<grid, block, 0, st>>>(a);
                else
                    dtrdt_step_kernel<true, 5, false><<<grid, block, 0, st>>>(a);
            } else if (packed) {
                OCT_LAUNCH(0, true);
            } else {
                OCT_LAUNCH(0, false);
            }
    }
#undef OCT_LAUNCH
    return cudaGetLastError();
}

cudaError_t launch_advance_t(uint32_t *t_ptr, cudaStream_t st) {
    advance_t_kernel<<<1, 1, 0, st>>>(t_ptr);
    return cudaGetLastError();
}

}  // namespace oct
