// Block layer of DTrDT with thread cells coarser than 4x4 sites: cx x cy
// sites, cx in {4, 8, 16, 32}, cy in {4, 8, 16} (the paper's TC=1,1 is 8x8,
// TC=2,1 16x8, TC=2,2 16x16, TC=3,2 32x16; Sec. 3.1.1).
//
// Lane layout: as for 4x4 cells, a lane holds 32 x 16 sites of the sub-tile
// (16 X-row and 16 Y-row words, the copies E, D of its right column and lower
// row), staged and written back by stage_lane / write_back.  A lane row holds
// 32/cx cells per TC row and 16/cy TC rows.
//
// Random streams follow the same reading as for 4x4 cells.  A group is four
// TC rows of one 32-site band column (g = group row * (Bx/32) + band column,
// TC row m = 0..3 inside it), so a group spans cy/4 lane rows:
//   set draw   (t, k|(s/64)<<2, T, SET<<28): word (s%64)/16, bits 2(s%16)..+1
//   site draw  (t, k|(s/spw)<<2, T, SITE<<28|g): word m, bits cx*j +
//              (s%spw)*(cx/spw) .. + bpt-1 for cell j of the band; the low
//              log2(cx/2) bits are the x offset inside the sub-cell, the next
//              log2(cy/2) the y offset (bpt = their sum, spw = 2 if 2 bpt <= cx)
//   acceptance bits 31..28 of the uniform of cell (j, m): bit
//              (s%SPL)*4*TPB + 4j+m of the four words of
//              (t, k|((s/SPL)*8)<<2, T, ACC<<28|g), SPL = cx/4 steps per
//              block (a group uses 4*TPB of the 32 positions per step);
//              bits 27..0, only for ties, from the group's tail stream in
//              order of position 4j+m.
// Because the positions 4j+m of one group interleave the lanes of the group
// (each holds some of its TC rows m), a tied candidate's place in the tail
// stream is the number of ties of the earlier groups plus the ties of its
// own group at lower positions, formed from the group's ties gathered by
// shuffles.
#pragma once
#include <cstdint>

#include "oct_internal.h"
#include "subtile.cuh"
#include "tiles.cuh"

namespace oct {

__host__ __device__ constexpr int ilog2c(int v) { return v <= 1 ? 0 : 1 + ilog2c(v / 2); }

template <int CX, int CY>
struct CellShape {
    static_assert((CX == 4 || CX == 8 || CX == 16 || CX == 32) && (CY == 4 || CY == 8 || CY == 16),
                  "thread cells of cx in {4,8,16,32} and cy in {4,8,16} sites");
    static constexpr int UX = CX / 2, UY = CY / 2;           // sub-cell
    static constexpr int BXB = ilog2c(UX), BYB = ilog2c(UY);  // random bits per offset
    static constexpr int BPT = BXB + BYB;
    static constexpr int TPB = 32 / CX;                      // cells per band (lane row)
    static constexpr int NTR = 16 / CY;                      // TC rows per lane
    static constexpr int GS = CY / 4;                        // lane rows per group
    static constexpr int SPW = (2 * BPT <= CX) ? 2 : 1;      // steps served by one site field
    static constexpr int SPL = CX / 4;                       // steps served by one level block
    static constexpr int STEPS = CX * CY;                    // collective steps per device step
    static constexpr uint32_t CMASK = CX == 32 ? 0xFFFFFFFFu : ((1u << CX) - 1u);
};

// Lane context of the coarse-cell block layer: c.g is the lane's group (for
// the site and acceptance streams); lane is its index inside the sub-tile
// (for the tail-stream refill); gr, gh its group row and lane row inside the
// group; m0 the TC row m of its first TC row.
struct CellCtx {
    LaneCtx c;
    int lane;
    int gr, gh;
    uint32_t m0;
};

__device__ __forceinline__ uint32_t word_of(const uint4 &w, uint32_t m) {
    return pick4(m, w.x, w.y, w.z, w.w);
}

// Phase 1 with sub-cell set (dx, DY): every cell (j, TC row i) of the lane
// attempts site (cx*j + dx*cx/2 + rx, i*cy + DY*cy/2 + ry) of the lane.  The
// cells' sites are gathered into one column mask per row of the active
// half (cand[i*UY + v] holds row i*cy + DY*UY + v); an attempt is eligible iff
// X(s) != X(s+x), Y(s) != Y(s+y) and X(s) == Y(s) (Eq. (1)), the minimum
// being X(s) = 0.  Candidates needing a draw are packed to bit 4j+m.
template <int CX, int CY, int DY, bool RANDOM, int SPEC>
__device__ __forceinline__ void cells_candidates(const uint32_t (&X)[16], const uint32_t (&Y)[16], uint32_t E,
                                                 uint32_t D, const uint4 &site, uint32_t s, uint32_t dx,
                                                 const CellCtx &cc, uint32_t (&cand)[8], uint32_t &pmin,
                                                 uint32_t &pmax) {
    using S = CellShape<CX, CY>;
    const uint32_t sub = (s % S::SPW) * (CX / S::SPW);
    pmin = 0u;
    pmax = 0u;
#pragma unroll
    for (int i = 0; i < S::NTR; ++i) {
        const uint32_t m = cc.m0 + static_cast<uint32_t>(i);
        const uint32_t u = word_of(site, m) >> sub;
        uint32_t M[S::UY];
#pragma unroll
        for (int v = 0; v < S::UY; ++v) M[v] = 0u;
#pragma unroll
        for (int j = 0; j < S::TPB; ++j) {
            const uint32_t f = (u >> (CX * j)) & ((1u << S::BPT) - 1u);
            const uint32_t rx = f & static_cast<uint32_t>(S::UX - 1), ry = f >> S::BXB;
            const uint32_t bit = 1u << (static_cast<uint32_t>(CX * j) + dx * S::UX + rx);
#pragma unroll
            for (int v = 0; v < S::UY; ++v) M[v] |= (ry == static_cast<uint32_t>(v)) ? bit : 0u;
        }
        uint32_t mn = 0u, mx = 0u;
#pragma unroll
        for (int v = 0; v < S::UY; ++v) {
            const int r = i * CY + DY * S::UY + v;
            const uint32_t x = X[r];
            const uint32_t xr = __funnelshift_r(x, E >> r, 1);
            const uint32_t y = Y[r];
            const uint32_t yd = (r + 1 < 16) ? Y[(r + 1) & 15] : D;
            uint32_t cd;
            if (SPEC == 1)
                cd = M[v] & ~x & xr & ~y & yd;  // deposition only: the minima
            else
                cd = M[v] & (x ^ xr) & (y ^ yd) & ~(x ^ y);
            cand[i * S::UY + v] = cd;
            if (RANDOM) {
                mn |= cd & ~x;
                mx |= cd & x;
            }
        }
        if (RANDOM) {
            if (SPEC != 2) {
                mn &= cc.c.p_random;
                mx &= cc.c.q_random;
            }
#pragma unroll
            for (int j = 0; j < S::TPB; ++j) {
                const uint32_t cm = S::CMASK << (CX * j);
                const uint32_t pos = 1u << (4u * static_cast<uint32_t>(j) + m);
                pmin |= (mn & cm) ? pos : 0u;
                pmax |= (mx & cm) ? pos : 0u;
            }
        }
    }
}

// Phase 2: acceptance of the lane's packed candidates (bit 4j+m), as in
// accept_candidates, for groups that span GS lane rows: a tied candidate's
// word in its group's tail stream is ranked among the ties of the whole group.
template <int GS>
__device__ __forceinline__ uint32_t cells_accept(uint32_t pmin, uint32_t pmax, const uint4 &W, const CellCtx &cc,
                                                 TailPool &tp) {
    const LaneCtx &c = cc.c;
    const uint32_t lw[4] = {W.x, W.y, W.z, W.w};
    uint32_t acc = 0, und = pmin | pmax;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const uint32_t bit = 31u - static_cast<uint32_t>(i);
        const uint32_t tb = (((c.thr_p >> bit) & 1u) ? pmin : 0u) | (((c.thr_q >> bit) & 1u) ? pmax : 0u);
        acc |= und & tb & ~lw[i];
        und &= ~(tb ^ lw[i]);
    }
    // ties of the lane's whole group (its GS lane rows)
    uint32_t gund = und;
    if (GS > 1) {
        gund = 0u;
#pragma unroll
        for (int h = 0; h < GS; ++h) {
            const int row = cc.gr * GS + h;
            const bool ok = row < c.GY;
            const int src = ok ? row * c.GX + c.gx : cc.lane;
            const uint32_t v = __shfl_sync(kFull, und, src);
            gund |= ok ? v : 0u;
        }
    }
    // The group's ties take the next words of its tail stream in order of
    // position; every lane of the group keeps the group's stream in its own
    // slot, so that it finds the words of its own ties there.
    if (__all_sync(kFull, gund == 0u)) return acc;
    const uint32_t ng = static_cast<uint32_t>(__popc(gund));
    tail_refill(ng, c.g, c, tp);
    // (w >> 4) < (P32 mod 2^28)  <=>  w < 16 (P32 mod 2^28)
    const uint32_t low_p = c.thr_p << 4, low_q = c.thr_q << 4;
    while (und) {
        const uint32_t bit = und & (0u - und);
        und ^= bit;
        const uint32_t at = tp.head + static_cast<uint32_t>(__popc(gund & (bit - 1u)));
        const uint32_t w = tp.ring[at & static_cast<uint32_t>(kRingWordsPerLane - 1)];
        acc |= (w < ((pmin & bit) ? low_p : low_q)) ? bit : 0u;
    }
    tp.head += ng;
    return acc;
}

// Phase 3 with sub-cell set (dx, DY): flips of the accepted candidates, then
// the exchange of the neighbour copies with the lanes right/left and
// below/above (flips reach bit 31 only for dx = 1, bit 0 only for dx = 0, row
// 15 only for DY = 1 and row 0 only for DY = 0).
template <int CX, int CY, int DY, bool RANDOM, int SPEC>
__device__ __forceinline__ void cells_apply(uint32_t (&X)[16], uint32_t (&Y)[16], uint32_t &E, uint32_t &D,
                                            uint32_t dx, uint32_t acc, const uint32_t (&cand)[8], const CellCtx &cc,
                                            int &net) {
    using S = CellShape<CX, CY>;
    const LaneCtx &c = cc.c;
    uint32_t dE = 0u, dB0 = 0u, dD = 0u, dY0 = 0u;
#pragma unroll
    for (int i = 0; i < S::NTR; ++i) {
        const uint32_t m = cc.m0 + static_cast<uint32_t>(i);
        uint32_t spread = 0u;
        if (RANDOM) {
#pragma unroll
            for (int j = 0; j < S::TPB; ++j)
                spread |= ((acc >> (4u * static_cast<uint32_t>(j) + m)) & 1u) ? (S::CMASK << (CX * j)) : 0u;
        }
        const uint32_t amin = c.p_always | (spread & c.p_random);
        const uint32_t amax = c.q_always | (spread & c.q_random);
#pragma unroll
        for (int v = 0; v < S::UY; ++v) {
            const int r = i * CY + DY * S::UY + v;
            const uint32_t x = X[r];
            const uint32_t cd = cand[i * S::UY + v];
            uint32_t f;
            if (SPEC == 1) {
                f = cd;
                net += __popc(f);
            } else if (SPEC == 2) {
                f = cd & spread;
            } else {
                f = cd & ((~x & amin) | (x & amax));
                net += always_net<RANDOM>(f, x, c);
            }
            X[r] = x ^ (f * 3u);  // f ^ (f << 1): one flip per cell, cells at least cx columns apart
            Y[r] ^= f;
            if (r + 1 < 16)
                Y[(r + 1) & 15] ^= f;
            else
                D ^= f;
            dE |= (f >> 31) << r;
            dB0 |= (f & 1u) << r;
            if (r == 15) dD = f;
            if (r == 0) dY0 = f;
        }
    }
    if (dx) {
        // flips at bit 31 changed column 0 of the right neighbour (this lane's E)
        E ^= dE;
        const uint32_t vr = __shfl_up_sync(kFull, dE, 1);
        if (c.gx > 0) {
#pragma unroll
            for (int i = 0; i < S::NTR; ++i)
#pragma unroll
                for (int v = 0; v < S::UY; ++v) {
                    const int r = i * CY + DY * S::UY + v;
                    X[r] ^= (vr >> r) & 1u;
                }
        }
    } else {
        // flips at bit 0 changed this lane's column 0, mirrored by the left neighbour's E
        const uint32_t vl = __shfl_down_sync(kFull, dB0, 1);
        if (c.gx < c.GX - 1) E ^= vl;
    }
    if (DY) {
        const uint32_t vd = __shfl_up_sync(kFull, dD, c.GX);  // row 16 (D) belongs to the lane below
        if (c.gy > 0) Y[0] ^= vd;
    } else {
        const uint32_t vu = __shfl_down_sync(kFull, dY0, c.GX);  // row 0 is mirrored by the lane above's D
        if (c.gy < c.GY - 1) D ^= vu;
    }
}

// Device step on one sub-tile with cx x cy-site thread cells: stage, the cx*cy
// single-hit collective steps, write back.  One sub-tile per warp.
template <int CX, int CY, bool RANDOM, int SPEC>
__device__ __forceinline__ void run_subtile_cells(uint32_t *lat, uint32_t L, uint32_t plane_rows, uint32_t wpr,
                                                  uint32_t Bx, uint32_t By,
                                                  uint32_t x0, uint32_t y0, bool active, const CellCtx &cc,
                                                  uint32_t *ring, int &net, int &draws, int &tails) {
    using S = CellShape<CX, CY>;
    const LaneCtx &c = cc.c;
    TailPool tp;
    tp.ring = ring + static_cast<uint32_t>(kRingWordsPerLane) * static_cast<uint32_t>(cc.lane);  // own slot
    tp.head = 0u;
    tp.end = 0u;
    tp.rounds = 0u;
    const LaneGeom q = lane_geom(lat, L, plane_rows, wpr, By, x0, y0, c);
    uint32_t X[16], Y[16], E, D;
    stage_lane(q, L, wpr, Bx, x0, active, c, X, Y, E, D);

    uint4 setw = make_uint4(0u, 0u, 0u, 0u), site = make_uint4(0u, 0u, 0u, 0u), lvl = make_uint4(0u, 0u, 0u, 0u);
    for (uint32_t s = 0; s < static_cast<uint32_t>(S::STEPS); ++s) {
        if ((s & 63u) == 0u) setw = philox4x32_10(c.t, c.k | ((s >> 6) << 2), c.T, kTagSet << 28, c.k0, c.k1);
        // the set, broadcast from lane 0 (all lanes drew the same one) so that the
        // branches on it are warp-uniform for the compiler
        const uint32_t d = __shfl_sync(kFull, (word_of(setw, (s >> 4) & 3u) >> (2u * (s & 15u))) & 3u, 0);
        if (s % S::SPW == 0u)
            site = philox4x32_10(c.t, c.k | ((s / S::SPW) << 2), c.T, (kTagSite << 28) | c.g, c.k0, c.k1);
        uint32_t cand[8], pmin, pmax;
        if (d & 2u)
            cells_candidates<CX, CY, 1, RANDOM, SPEC>(X, Y, E, D, site, s, d & 1u, cc, cand, pmin, pmax);
        else
            cells_candidates<CX, CY, 0, RANDOM, SPEC>(X, Y, E, D, site, s, d & 1u, cc, cand, pmin, pmax);
        uint32_t acc = 0u;
        if (RANDOM) {
            draws += __popc(pmin | pmax);
            if (s % S::SPL == 0u)
                lvl = philox4x32_10(c.t, c.k | (((s / S::SPL) * 8u) << 2), c.T, (kTagAcc << 28) | c.g, c.k0, c.k1);
            const uint32_t sh = (s % S::SPL) * 4u * S::TPB;  // this step's positions
            const uint4 W = make_uint4(lvl.x >> sh, lvl.y >> sh, lvl.z >> sh, lvl.w >> sh);
            acc = cells_accept<S::GS>(pmin, pmax, W, cc, tp);
            net += random_net(acc, pmin, pmax);
        }
        if (d & 2u)
            cells_apply<CX, CY, 1, RANDOM, SPEC>(X, Y, E, D, d & 1u, acc, cand, cc, net);
        else
            cells_apply<CX, CY, 0, RANDOM, SPEC>(X, Y, E, D, d & 1u, acc, cand, cc, net);
    }
    write_back<false>(q, L, wpr, active, c, X, Y, E, D);
    tails = static_cast<int>(tp.rounds);
}

// One device step with cx x cy-site cells: the kernel and its launch.  The
// launch functions are instantiated in cells_*.cu, a few shapes per
// translation unit so that they compile in parallel.
// Device layer as for 4x4 cells (Sec. 3, DTr): the origin (ox, oy) and the
// set permutation come from Philox(t, 0, 0, MCS<<28) once per MCS; sub-tile T
// of set sigma = perm[k] starts at (ox + 2Bx tx + Bx (sigma&1), oy + 2By ty +
// By (sigma>>1)) mod L.
template <int CX, int CY, bool RANDOM, int SPEC>
__global__ void __launch_bounds__(kStepWarpsPerBlock * 32, kStepBlocksPerSMPacked)
    cells_step_kernel(const StepArgs a) {
    using S = CellShape<CX, CY>;
    __shared__ __align__(16) uint32_t ring[kStepWarpsPerBlock * 32 * kRingWordsPerLane];
    const int lane = threadIdx.x & 31;
    const uint32_t w = blockIdx.x * kStepWarpsPerBlock + (threadIdx.x >> 5);
    if (w >= work_tiles(a)) return;  // the whole warp leaves together

    const uint32_t t = *a.t_ptr;
    const uint32_t L = a.L;
    const TilePlace pl = place_tile(a, w, t);
    const uint32_t T = pl.T, x0 = pl.x0, y0 = pl.y0;

    CellCtx cc;
    LaneCtx &c = cc.c;
    c.GX = static_cast<int>(a.GX);
    c.GY = static_cast<int>(a.GY);
    c.gx = lane % c.GX;
    c.gy = lane / c.GX;
    const uint32_t G = a.GX * a.GY;
    const bool active = static_cast<uint32_t>(lane) < G;
    c.active = active;
    c.last = static_cast<int>(G - 1u);
    c.t = t;
    c.k = a.k;
    c.T = T;
    c.k0 = a.k0;
    c.k1 = a.k1;
    c.thr_p = a.thr_p;
    c.thr_q = a.thr_q;
    c.p_always = a.p_always;
    c.q_always = a.q_always;
    c.p_random = a.p_random;
    c.q_random = a.q_random;
    cc.lane = lane;
    cc.gr = c.gy / S::GS;
    cc.gh = c.gy % S::GS;
    cc.m0 = static_cast<uint32_t>(cc.gh * S::NTR);
    c.g = static_cast<uint32_t>(cc.gr * c.GX + c.gx);  // the lane's group

    int net = 0, draws = 0, tails = 0;
    run_subtile_cells<CX, CY, RANDOM, SPEC>(a.lat, L, a.plane_rows, a.wpr, a.Bx, a.By, x0, y0, active, cc,
                                            ring + (threadIdx.x >> 5) * 32 * kRingWordsPerLane, net, draws,
                                            tails);

    const int total = __reduce_add_sync(kFull, net);
    if (lane == 0 && total != 0)
        atomicAdd(&a.net[T % kNetSlots], static_cast<unsigned long long>(static_cast<long long>(total)));
    if (RANDOM) {
        const unsigned nd = __reduce_add_sync(kFull, static_cast<unsigned>(draws));
        if (lane == 0 && nd != 0u) atomicAdd(&a.draws[T % kNetSlots], static_cast<unsigned long long>(nd));
        // tail-stream Philox blocks stored by the sub-tile's lanes
        const unsigned nb = __reduce_add_sync(kFull, active ? static_cast<unsigned>(tails) : 0u);
        if (lane == 0 && nb != 0u) atomicAdd(&a.tails[T % kNetSlots], static_cast<unsigned long long>(nb));
    }
}

template <int CX, int CY>
void launch_cells_shape(const StepArgs &a, bool any_random, const dim3 &grid, const dim3 &block, cudaStream_t st) {
    if (!any_random && a.p_always == 0xFFFFFFFFu && a.q_always == 0u)
        cells_step_kernel<CX, CY, false, 1><<<grid, block, 0, st>>>(a);  // deposition only (p = 1, q = 0)
    else if (any_random && a.p_random && a.q_random)
        cells_step_kernel<CX, CY, true, 2><<<grid, block, 0, st>>>(a);   // both rates inside (0, 1)
    else if (any_random)
        cells_step_kernel<CX, CY, true, 0><<<grid, block, 0, st>>>(a);
    else
        cells_step_kernel<CX, CY, false, 0><<<grid, block, 0, st>>>(a);
}

}  // namespace oct
