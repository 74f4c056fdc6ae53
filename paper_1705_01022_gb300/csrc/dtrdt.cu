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
// GB300 mapping.  One warp owns one sub-tile for the whole device step; no
// block-wide barrier is needed.  Lane (gx, gy) holds a group of 32 x 16 sites
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

namespace oct {
namespace {

template <bool RANDOM, int SCHEME>
__global__ void __launch_bounds__(kStepWarpsPerBlock * 32, kStepBlocksPerSM)
    dtrdt_step_kernel(const StepArgs a) {
    __shared__ __align__(16) uint32_t ring[kStepWarpsPerBlock * 32 * kRingWordsPerLane];
    const int lane = threadIdx.x & 31;
    const uint32_t T = blockIdx.x * kStepWarpsPerBlock + (threadIdx.x >> 5);
    if (T >= a.tiles_x * a.tiles_y) return;  // the whole warp leaves together

    const uint32_t t = *a.t_ptr;
    const uint32_t L = a.L;
    // Device layer: origin and set order of this MCS (same for every warp).
    const uint4 M = philox4x32_10(t, 0u, 0u, kTagMcs << 28, a.k0, a.k1);
    const uint32_t ox = static_cast<uint32_t>((static_cast<uint64_t>(M.x) * L) >> 32);
    const uint32_t oy = static_cast<uint32_t>((static_cast<uint64_t>(M.y) * L) >> 32);
    const uint32_t pidx = static_cast<uint32_t>((static_cast<uint64_t>(M.z) * 24u) >> 32);
    const int sigma = perm_element(pidx, a.k);
    const uint32_t tx = T % a.tiles_x, ty = T / a.tiles_x;
    const uint32_t x0 = static_cast<uint32_t>(
        (static_cast<uint64_t>(ox) + 2ull * a.Bx * tx + static_cast<uint64_t>(a.Bx) * (sigma & 1)) % L);
    const uint32_t y0 = static_cast<uint32_t>(
        (static_cast<uint64_t>(oy) + 2ull * a.By * ty + static_cast<uint64_t>(a.By) * (sigma >> 1)) % L);

    LaneCtx c;
    c.GX = static_cast<int>(a.GX);
    c.GY = static_cast<int>(a.GY);
    c.gx = lane % c.GX;
    c.gy = lane / c.GX;
    const bool active = c.gy < c.GY;
    c.active = active;
    c.last = c.GX * c.GY - 1;
    c.t = t;
    c.k = a.k;
    c.T = T;
    c.g = static_cast<uint32_t>(c.gy * c.GX + c.gx);
    c.k0 = a.k0;
    c.k1 = a.k1;
    c.thr_p = a.thr_p;
    c.thr_q = a.thr_q;
    c.p_always = a.p_always;
    c.q_always = a.q_always;
    c.p_random = a.p_random;
    c.q_random = a.q_random;

    const uint32_t wpr = a.wpr;
    int net = 0, draws = 0;
    run_subtile<RANDOM, false, SCHEME>(a.lat, L, wpr, a.Bx, a.By, x0, y0, active, c,
                               ring + (threadIdx.x >> 5) * 32 * kRingWordsPerLane, net, draws);

    // Net flips (and acceptance draws): one atomic per warp into a spread of counters.
    const int total = __reduce_add_sync(kFull, net);
    if (lane == 0 && total != 0)
        atomicAdd(&a.net[T % kNetSlots], static_cast<unsigned long long>(static_cast<long long>(total)));
    if (RANDOM) {
        const unsigned nd = __reduce_add_sync(kFull, static_cast<unsigned>(draws));
        if (lane == 0 && nd != 0u) atomicAdd(&a.draws[T % kNetSlots], static_cast<unsigned long long>(nd));
    }
}

__global__ void advance_t_kernel(uint32_t *t_ptr) { *t_ptr += 1u; }

}  // namespace

cudaError_t launch_dtrdt_step(const StepArgs &a, bool any_random, cudaStream_t st) {
    const uint32_t n_tiles = a.tiles_x * a.tiles_y;
    const uint32_t blocks = (n_tiles + kStepWarpsPerBlock - 1) / kStepWarpsPerBlock;
    const dim3 grid(blocks), block(kStepWarpsPerBlock * 32);
    switch (a.scheme) {
        case 1:
            if (any_random)
                dtrdt_step_kernel<true, 1><<<grid, block, 0, st>>>(a);
            else
                dtrdt_step_kernel<false, 1><<<grid, block, 0, st>>>(a);
            break;
        case 2:
            if (any_random)
                dtrdt_step_kernel<true, 2><<<grid, block, 0, st>>>(a);
            else
                dtrdt_step_kernel<false, 2><<<grid, block, 0, st>>>(a);
            break;
        case 3:
            if (any_random)
                dtrdt_step_kernel<true, 3><<<grid, block, 0, st>>>(a);
            else
                dtrdt_step_kernel<false, 3><<<grid, block, 0, st>>>(a);
            break;
        default:
            if (any_random)
                dtrdt_step_kernel<true, 0><<<grid, block, 0, st>>>(a);
            else
                dtrdt_step_kernel<false, 0><<<grid, block, 0, st>>>(a);
    }
    return cudaGetLastError();
}

cudaError_t launch_advance_t(uint32_t *t_ptr, cudaStream_t st) {
    advance_t_kernel<<<1, 1, 0, st>>>(t_ptr);
    return cudaGetLastError();
}

}  // namespace oct
