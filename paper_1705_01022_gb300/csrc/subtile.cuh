// Device code shared by the plain and the batched device-step kernels: one
// device step on a sub-tile held by warp lanes, with the block layer of
// DTrDT, DTrDB or DTrDTr (see dtrdt.cu for the method and the lane layout).
// Streams beyond those listed in dtrdt.cu: DTrDB draws a site of the whole
// cell from (t, k|s<<2, T, SITE_DB<<28|g), DTrDTr its block-layer origin from
// (t, k, T, BORG<<28), byte s of the device step.
#pragma once
#include <cstdint>

#include "philox.cuh"

namespace oct {

constexpr uint32_t kFull = 0xFFFFFFFFu;
constexpr uint32_t kNib = 0x11111111u;  // bit 0 of every 4-bit TC column

// Element k of the idx-th permutation of (0,1,2,3) in lexicographic order.
__device__ __forceinline__ int perm_element(uint32_t idx, uint32_t k) {
    uint32_t remaining = 0x3210u;  // nibbles: the symbols not used yet, in order
    uint32_t radix = 6u;            // (3 - i)!
    int e = 0;
    for (uint32_t i = 0; i <= k; ++i) {
        const uint32_t pick = idx / radix;
        idx -= pick * radix;
        e = static_cast<int>((remaining >> (4u * pick)) & 0xFu);
        const uint32_t low = remaining & ((1u << (4u * pick)) - 1u);
        const uint32_t high = remaining >> (4u * (pick + 1u));
        remaining = low | (high << (4u * pick));
        radix = (i == 0) ? 2u : 1u;
    }
    return e;
}

// Sets the bits of *w selected by mask to those of v, leaving the others, as
// two reductions (no value returned, so the warp does not wait for them).
__device__ __forceinline__ void reduce_bits(uint32_t *w, uint32_t v, uint32_t mask) {
    atomicAnd(w, v | ~mask);
    atomicOr(w, v & mask);
}

struct LaneCtx {
    uint32_t t, k, T, g;
    uint32_t k0, k1;
    uint32_t thr_p, thr_q;
    uint32_t p_always, q_always, p_random, q_random;
    int gx, gy, GX, GY;
    int last;      // lane holding the sub-tile's last group
    bool active;   // this lane holds a group of a sub-tile
};

// Net flips (depositions minus removals) among the flips f of one row (x: the
// row's X bits before the flips) that were accepted without a draw (p = 1 or
// q = 1).  Flips decided by a draw are counted once per step from the packed
// acceptance bits instead (random_net).
template <bool RANDOM>
__device__ __forceinline__ int always_net(uint32_t f, uint32_t x, const LaneCtx &c) {
    if (RANDOM) {
        if ((c.p_always | c.q_always) == 0u) return 0;
        return __popc(f & ~x & c.p_always) - __popc(f & x & c.q_always);
    }
    if (c.q_always == 0u) return __popc(f);   // only depositions are possible
    if (c.p_always == 0u) return -__popc(f);  // only removals
    return __popc(f & ~x) - __popc(f & x);
}

// Net flips among the packed candidates accepted by their draw.
__device__ __forceinline__ int random_net(uint32_t acc, uint32_t pmin, uint32_t pmax) {
    return __popc(acc & pmin) - __popc(acc & pmax);
}

// Tail words read at once for the first ties (accept_candidates), per block
// layer, as measured at L=2^17: DTrDT on full warps gains 2.6 % from three;
// on packed warps, in DTrDB (three acceptance passes per step, often with
// few ties) and in DTrDTr the loop alone is as fast or faster.
constexpr int kPreDt = 3, kPrePacked = 0, kPreDb = 0, kPreDtr = 0;

// Each lane keeps its group's tail stream (see accept_candidates) in its own
// slot of kRingWordsPerLane words of shared memory, a ring above the live
// window: fewer than (ties of one step, at most 32) + 4 words.
constexpr int kRingWordsPerLane = 64;

struct TailPool {
    uint32_t *ring;  // the lane's own slot of kRingWordsPerLane words
    uint32_t head;   // words of the group's tail stream used so far in this device step
    uint32_t end;    // words generated into the slot so far in this device step
    uint32_t rounds; // Philox blocks the lane generated into its slot
};

// Tops up the lane's slot until it holds the `need` words after head; every
// lane of the warp takes part in each round (one Philox block per lane, block
// end/4 of its group's stream, kept only if the slot has room).
__device__ __forceinline__ void tail_refill(uint32_t need, uint32_t g, const LaneCtx &c, TailPool &tp) {
    while (__any_sync(kFull, tp.end < tp.head + need)) {
        const uint4 B = philox4x32_10(c.t, c.k | ((tp.end >> 2) << 2), c.T, (kTagTail << 28) | g, c.k0, c.k1);
        if (tp.end - tp.head <= static_cast<uint32_t>(kRingWordsPerLane - 4)) {
            *reinterpret_cast<uint4 *>(tp.ring + (tp.end & static_cast<uint32_t>(kRingWordsPerLane - 1))) = B;
            tp.end += 4u;
            ++tp.rounds;
        }
    }
}

// Acceptance of the packed candidates (bit 4j+m = thread cell column j, TC
// row m).  The uniform u of a candidate, most significant bit first:
//  * bits 31..28 come from the four level words of the lane's group (bit
//    4j+m of word l is bit 31-l), one Philox block per step; all 32 thread
//    cells of the lane are compared with P32 together, one level at a time;
//    the comparison is decided unless the four bits equal P32's;
//  * a candidate still tied takes its bits 27..0 from the top of the next word
//    of its group's tail stream (word i = word i%4 of Philox(t, k|(i/4)<<2, T,
//    TAIL<<28|g), counted from 0 each device step), the group's ties of a step
//    in order of position.  A lane holds one group, so it takes its own words.
__device__ __forceinline__ uint4 level_words(uint32_t s, const LaneCtx &c) {
    return philox4x32_10(c.t, c.k | ((s * 8u) << 2), c.T, (kTagAcc << 28) | c.g, c.k0, c.k1);
}

// PRE: tail words the lane reads at once for its first ties (0: one word per
// tie in the loop); the fastest choice differs between the block layers.
template <int PRE>
__device__ __forceinline__ uint32_t accept_candidates(uint32_t pmin, uint32_t pmax, const uint4 &W,
                                                      const LaneCtx &c, TailPool &tp) {
    const uint32_t lw[4] = {W.x, W.y, W.z, W.w};
    uint32_t acc = 0, und = pmin | pmax;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const uint32_t bit = 31u - static_cast<uint32_t>(i);
        const uint32_t tb = (((c.thr_p >> bit) & 1u) ? pmin : 0u) | (((c.thr_q >> bit) & 1u) ? pmax : 0u);
        acc |= und & tb & ~lw[i];
        und &= ~(tb ^ lw[i]);
    }
    // Skip the tail stage only when no lane of the warp needs it: every lane
    // takes part in the refill rounds.
    if (__all_sync(kFull, und == 0u)) return acc;
    const uint32_t nt = static_cast<uint32_t>(__popc(und));
    tail_refill(nt, c.g, c, tp);
    // (w >> 4) < (P32 mod 2^28)  <=>  w < 16 (P32 mod 2^28)
    const uint32_t low_p = c.thr_p << 4, low_q = c.thr_q << 4;
    // The lane's next PRE tail words are read at once and its first PRE ties
    // decided without a branch (a lane has fewer than one tie per step on
    // average); further ties take the loop, one word each.
    constexpr uint32_t kMask = static_cast<uint32_t>(kRingWordsPerLane - 1);
    const uint32_t h = tp.head;
    if (PRE > 0) {
        uint32_t wp[PRE > 0 ? PRE : 1];
#pragma unroll
        for (int j = 0; j < PRE; ++j) wp[j] = tp.ring[(h + static_cast<uint32_t>(j)) & kMask];
#pragma unroll
        for (int j = 0; j < PRE; ++j) {
            const uint32_t bit = und & (0u - und);  // lowest tied position (0 once none is left)
            und ^= bit;
            acc |= (wp[j] < ((pmin & bit) ? low_p : low_q)) ? bit : 0u;
        }
    }
    uint32_t hn = h + static_cast<uint32_t>(PRE);
    while (und) {
        const uint32_t bit = und & (0u - und);
        und ^= bit;
        const uint32_t w = tp.ring[hn & kMask];
        ++hn;
        acc |= (w < ((pmin & bit) ? low_p : low_q)) ? bit : 0u;
    }
    tp.head = h + nt;
    return acc;
}

// A collective step runs in three phases: the candidates of every thread
// cell of the lane (specialised on the set's row offset dy), the acceptance
// draws (one copy of the code, shared by both offsets), and the flips with
// the neighbour exchange (specialised again).
//
// Phase 1 with sub-cell set (dx, DY).  X/Y hold the lane's 16 rows, E bit r
// the X bit just right of row r, D the Y row just below row 15.  An attempt at
// s is eligible iff X(s) != X(s+x), Y(s) != Y(s+y) and X(s) == Y(s): then
// X(s) = 0 is the minimum of Eq. (1), X(s) = 1 the maximum.  Candidates that
// need an acceptance draw are packed to bit 4j+m (TC column j, TC row m).
// SPEC 1 (deposition only: p = 1, q = 0, the KPZ case): every eligible
// minimum flips and no maximum does, so the candidates are the minima
// themselves.  SPEC 2 (both 0 < p < 1 and 0 < q < 1): every candidate needs a
// draw, so no always/never masks are applied.
template <int DY, bool RANDOM, int SPEC = 0>
__device__ __forceinline__ void step_candidates(const uint32_t (&X)[16], const uint32_t (&Y)[16],
                                                uint32_t E, uint32_t D, const uint4 &site, uint32_t s,
                                                uint32_t dx, const LaneCtx &c, uint32_t (&cnd0)[4],
                                                uint32_t (&cnd1)[4], uint32_t &pmin, uint32_t &pmax) {
    const uint32_t sw[4] = {site.x, site.y, site.z, site.w};
    const uint32_t sh2 = 2u * dx;
    pmin = 0u;
    pmax = 0u;
#pragma unroll
    for (int m = 0; m < 4; ++m) {
        // Site draw: bit 4j = x offset, bit 4j+1 = y offset of TC column j (for odd
        // steps run_subtile has shifted the words down to the step's field).
        const uint32_t u = sw[m];
        const uint32_t col = ((u & kNib) + kNib) << sh2;  // 1 + xoff: one-hot, no carries
        // the y offset, spread over the two columns col can take (bits 2dx, 2dx+1)
        const uint32_t yoff = dx ? (u & (kNib << 1)) * 6u : ((u >> 1) & kNib) * 3u;
        const int r0 = 4 * m + 2 * DY, r1 = r0 + 1;
        const uint32_t xa = X[r0], xb = X[r1];
        const uint32_t xra = __funnelshift_r(xa, E >> r0, 1);
        const uint32_t xrb = __funnelshift_r(xb, E >> r1, 1);
        const uint32_t ya = Y[r0], yb = Y[r1];
        const uint32_t yc = (r1 + 1 < 16) ? Y[(r1 + 1) & 15] : D;
        if (SPEC == 1) {
            // minimum: X(s) = 0, X(s+x) = 1, Y(s) = 0, Y(s+y) = 1
            cnd0[m] = col & ~yoff & ~xa & xra & ~ya & yb;
            cnd1[m] = col & yoff & ~xb & xrb & ~yb & yc;
            continue;
        }
        cnd0[m] = col & ~yoff & (xa ^ xra) & (ya ^ yb) & ~(xa ^ ya);
        cnd1[m] = col & yoff & (xb ^ xrb) & (yb ^ yc) & ~(xb ^ yb);
        if (RANDOM && SPEC == 2) {
            const uint32_t cc = cnd0[m] | cnd1[m];
            const uint32_t mx = (cnd0[m] & xa) | (cnd1[m] & xb);
            pmin |= (((cc * 3u) >> (sh2 + 1u)) & kNib) << m;
            pmax |= (((mx * 3u) >> (sh2 + 1u)) & kNib) << m;
        } else if (RANDOM) {
            const uint32_t mn = (cnd0[m] & ~xa) | (cnd1[m] & ~xb);
            const uint32_t mx = (cnd0[m] & xa) | (cnd1[m] & xb);
            const uint32_t cmn = SPEC == 2 ? mn : mn & c.p_random, cmx = SPEC == 2 ? mx : mx & c.q_random;
            // a cell has at most one candidate, at bit 4j + sh2 + xoff: 3 cmn sets bit
            // 4j + sh2 + 1 for either xoff (no carries: candidates are >= 3 bits apart)
            pmin |= (((cmn * 3u) >> (sh2 + 1u)) & kNib) << m;
            pmax |= (((cmx * 3u) >> (sh2 + 1u)) & kNib) << m;
        }
    }
    if (RANDOM && SPEC == 2) pmin &= ~pmax;  // pmin held every candidate: keep the minima
}

// Phase 3 with sub-cell set (dx, DY): flips of the accepted candidates (acc:
// packed acceptance bits) and the exchange with the neighbouring lanes.
template <int DY, bool RANDOM, int SPEC = 0>
__device__ __forceinline__ void step_apply(uint32_t (&X)[16], uint32_t (&Y)[16], uint32_t &E, uint32_t &D,
                                           uint32_t dx, uint32_t acc, const uint32_t (&cnd0)[4],
                                           const uint32_t (&cnd1)[4], const LaneCtx &c, int &net) {
    uint32_t f0s[4], f1s[4];
#pragma unroll
    for (int m = 0; m < 4; ++m) {
        const int r0 = 4 * m + 2 * DY, r1 = r0 + 1;
        uint32_t amin = c.p_always, amax = c.q_always, spread = 0u;
        if (RANDOM) {
            spread = ((acc >> m) & kNib) * 0xFu;
            amin |= spread & c.p_random;
            amax |= spread & c.q_random;
        }
        const uint32_t xa = X[r0], xb = X[r1];
        // accepted minima are where the candidate has X(s) = 0
        uint32_t f0, f1;
        if (SPEC == 1) {
            f0 = cnd0[m];
            f1 = cnd1[m];
            net += __popc(f0 | f1);  // a thread cell flips in one of the two rows
        } else if (SPEC == 2) {
            f0 = cnd0[m] & spread;  // the draw decides every candidate
            f1 = cnd1[m] & spread;
        } else {
            f0 = cnd0[m] & ((~xa & amin) | (xa & amax));
            f1 = cnd1[m] & ((~xb & amin) | (xb & amax));
            net += always_net<RANDOM>(f0, xa, c) + always_net<RANDOM>(f1, xb, c);
        }
        // f ^ (f << 1) = 3f: a cell flips at most one site, so flips are at
        // least three columns apart and the sum has no carries (FMA pipe)
        X[r0] = xa ^ (f0 * 3u);
        X[r1] = xb ^ (f1 * 3u);
        Y[r0] ^= f0;
        Y[r1] ^= f0 ^ f1;
        if (r1 + 1 < 16)
            Y[(r1 + 1) & 15] ^= f1;
        else
            D ^= f1;
        f0s[m] = f0;
        f1s[m] = f1;
    }

    // Keep the neighbour copies consistent (dx is uniform over the warp here).
    if (dx) {
        // Flips at bit 31 changed column 0 of the right neighbour (this lane's E).
        uint32_t dE = 0;
#pragma unroll
        for (int m = 0; m < 4; ++m) {
            const int r0 = 4 * m + 2 * DY;
            dE |= ((f0s[m] >> 31) << r0) | ((f1s[m] >> 31) << (r0 + 1));
        }
        E ^= dE;
        const uint32_t v = __shfl_up_sync(kFull, dE, 1);
        if (c.gx > 0) {
#pragma unroll
            for (int m = 0; m < 4; ++m) {
                const int r0 = 4 * m + 2 * DY, r1 = r0 + 1;
                X[r0] ^= (v >> r0) & 1u;
                X[r1] ^= (v >> r1) & 1u;
            }
        }
    } else {
        // Flips at bit 0 changed this lane's column 0, mirrored by the left neighbour's E.
        uint32_t dB0 = 0;
#pragma unroll
        for (int m = 0; m < 4; ++m) {
            const int r0 = 4 * m + 2 * DY;
            dB0 |= ((f0s[m] & 1u) << r0) | ((f1s[m] & 1u) << (r0 + 1));
        }
        const uint32_t v = __shfl_down_sync(kFull, dB0, 1);
        if (c.gx < c.GX - 1) E ^= v;
    }
    if (DY) {
        // Row 16 (D) belongs to the lane below.
        const uint32_t v = __shfl_up_sync(kFull, f1s[3], c.GX);
        if (c.gy > 0) Y[0] ^= v;
    } else {
        // Row 0 is mirrored by the lane above in its D.
        const uint32_t v = __shfl_down_sync(kFull, f0s[0], c.GX);
        if (c.gy < c.GY - 1) D ^= v;
    }
}

// The same two phases when the lanes of one warp belong to different
// sub-tiles, each with its own set draw: the row offset dy is a run-time value
// per lane (rows picked with selects instead of branches), and every shuffle
// runs unconditionally so that all 32 lanes take part.
template <bool RANDOM, int SPEC = 0>
__device__ __forceinline__ void step_candidates_rt(const uint32_t (&X)[16], const uint32_t (&Y)[16],
                                                   uint32_t E, uint32_t D, const uint4 &site, uint32_t s,
                                                   uint32_t dx, uint32_t dy, const LaneCtx &c,
                                                   uint32_t (&cnd0)[4], uint32_t (&cnd1)[4],
                                                   uint32_t &pmin, uint32_t &pmax) {
    const uint32_t sw[4] = {site.x, site.y, site.z, site.w};
    const uint32_t sh2 = 2u * dx;  // site words: shifted to the step's field by run_subtile
    const uint32_t ro = 2u * dy;
    pmin = 0u;
    pmax = 0u;
#pragma unroll
    for (int m = 0; m < 4; ++m) {
        const uint32_t u = sw[m];
        const uint32_t col = ((u & kNib) + kNib) << sh2;  // 1 + xoff: one-hot, no carries
        const uint32_t yoff = ((u >> 1) & kNib) * 0xFu;
        const uint32_t xa = dy ? X[4 * m + 2] : X[4 * m];
        const uint32_t xb = dy ? X[4 * m + 3] : X[4 * m + 1];
        const uint32_t ya = dy ? Y[4 * m + 2] : Y[4 * m];
        const uint32_t yb = dy ? Y[4 * m + 3] : Y[4 * m + 1];
        const uint32_t yc = dy ? (m < 3 ? Y[(4 * m + 4) & 15] : D) : Y[4 * m + 2];
        const uint32_t r0 = 4u * m + ro;
        const uint32_t xra = __funnelshift_r(xa, E >> r0, 1);
        const uint32_t xrb = __funnelshift_r(xb, E >> (r0 + 1u), 1);
        if (SPEC == 1) {
            cnd0[m] = col & ~yoff & ~xa & xra & ~ya & yb;  // the minima
            cnd1[m] = col & yoff & ~xb & xrb & ~yb & yc;
            continue;
        }
        cnd0[m] = col & ~yoff & (xa ^ xra) & (ya ^ yb) & ~(xa ^ ya);
        cnd1[m] = col & yoff & (xb ^ xrb) & (yb ^ yc) & ~(xb ^ yb);
        if (RANDOM) {
            const uint32_t mn = (cnd0[m] & ~xa) | (cnd1[m] & ~xb);
            const uint32_t mx = (cnd0[m] & xa) | (cnd1[m] & xb);
            const uint32_t cmn = SPEC == 2 ? mn : mn & c.p_random, cmx = SPEC == 2 ? mx : mx & c.q_random;
            pmin |= (((cmn * 3u) >> (sh2 + 1u)) & kNib) << m;  // see step_candidates
            pmax |= (((cmx * 3u) >> (sh2 + 1u)) & kNib) << m;
        }
    }
}

template <bool RANDOM, int SPEC = 0>
__device__ __forceinline__ void step_apply_rt(uint32_t (&X)[16], uint32_t (&Y)[16], uint32_t &E, uint32_t &D,
                                              uint32_t dy, uint32_t acc, const uint32_t (&cnd0)[4],
                                              const uint32_t (&cnd1)[4], const LaneCtx &c, int &net) {
    const uint32_t ro = 2u * dy;
    const uint32_t dym = dy ? 0xFFFFFFFFu : 0u;
    uint32_t dE = 0, dB0 = 0, dD = 0, dY0 = 0;
    uint32_t g0[4], g1[4];
#pragma unroll
    for (int m = 0; m < 4; ++m) {
        uint32_t amin = c.p_always, amax = c.q_always, spread = 0u;
        if (RANDOM) {
            spread = ((acc >> m) & kNib) * 0xFu;
            amin |= spread & c.p_random;
            amax |= spread & c.q_random;
        }
        uint32_t f0, f1;
        if (SPEC == 1) {
            f0 = cnd0[m];
            f1 = cnd1[m];
            net += __popc(f0 | f1);
        } else if (SPEC == 2) {
            f0 = cnd0[m] & spread;
            f1 = cnd1[m] & spread;
        } else {
            const uint32_t xa = dy ? X[4 * m + 2] : X[4 * m];
            const uint32_t xb = dy ? X[4 * m + 3] : X[4 * m + 1];
            f0 = cnd0[m] & ((~xa & amin) | (xa & amax));
            f1 = cnd1[m] & ((~xb & amin) | (xb & amax));
            net += always_net<RANDOM>(f0, xa, c) + always_net<RANDOM>(f1, xb, c);
        }
        g0[m] = f0 * 3u;  // 3f = f ^ (f << 1), see step_apply; applied after the exchange
        g1[m] = f1 * 3u;
        const uint32_t f01 = f0 ^ f1;
        Y[4 * m] ^= f0 & ~dym;
        Y[4 * m + 1] ^= f01 & ~dym;
        Y[4 * m + 2] ^= (f0 & dym) | (f1 & ~dym);
        Y[4 * m + 3] ^= f01 & dym;
        if (m < 3)
            Y[(4 * m + 4) & 15] ^= f1 & dym;
        else
            D ^= f1 & dym;
        dE |= ((f0 >> 31) << (4 * m)) | ((f1 >> 31) << (4 * m + 1));
        dB0 |= ((f0 & 1u) << (4 * m)) | ((f1 & 1u) << (4 * m + 1));
        if (m == 3) dD = f1 & dym;
        if (m == 0) dY0 = f0 & ~dym;
    }
    if (c.GX > 1) {  // warp-uniform: every sub-tile of a warp has the same shape
        dE <<= ro;
        dB0 <<= ro;
        E ^= dE;
        uint32_t vr = __shfl_up_sync(kFull, dE, 1);
        const uint32_t vl = __shfl_down_sync(kFull, dB0, 1);
        vr = c.gx > 0 ? (vr >> ro) : 0u;  // the left lane is in the same sub-tile: same row offset
#pragma unroll
        for (int m = 0; m < 4; ++m) {
            g0[m] ^= (vr >> (4 * m)) & 1u;
            g1[m] ^= (vr >> (4 * m + 1)) & 1u;
        }
        if (c.gx < c.GX - 1) E ^= vl;
    } else {
        E ^= dE << ro;
    }
#pragma unroll
    for (int m = 0; m < 4; ++m) {
        X[4 * m] ^= g0[m] & ~dym;
        X[4 * m + 1] ^= g1[m] & ~dym;
        X[4 * m + 2] ^= g0[m] & dym;
        X[4 * m + 3] ^= g1[m] & dym;
    }
    const uint32_t vd = __shfl_up_sync(kFull, dD, c.GX);
    const uint32_t vu = __shfl_down_sync(kFull, dY0, c.GX);
    if (c.gy > 0) Y[0] ^= vd;
    if (c.gy < c.GY - 1) D ^= vu;
}

// One collective step of single-hit DB (dead border) with 4 x 4-site thread
// cells: every cell attempts a uniform site of the whole cell (site word m:
// bits 4j, 4j+1 = x offset, 4j+2, 4j+3 = y offset of cell j in TC row m).
// The cell's border is its last column (x = 3) and last row (y = 3), where
// an update reaches the next cell.  DELAYED (both p and q non-zero): bulk
// attempts, then border attempts, then corner attempts, each phase decided on
// the state the earlier phases left; otherwise all attempts of the step are
// decided on the state before the step, which with one rate zero never lets
// two accepted flips meet.  Every candidate of a phase is found before any of
// its flips is applied.
// SPEC as for step_candidates: 1 deposition only, 2 both rates random.
template <bool RANDOM, bool DELAYED, int SPEC = 0>
__device__ __forceinline__ void db_step(uint32_t (&X)[16], uint32_t (&Y)[16], uint32_t &E, uint32_t &D,
                                        const uint4 &site, uint32_t s, const LaneCtx &c, TailPool &tp,
                                        int &net, int &draws) {
    const uint32_t sw[4] = {site.x, site.y, site.z, site.w};
    uint32_t sel[16];
#pragma unroll
    for (int m = 0; m < 4; ++m) {
        const uint32_t u = sw[m];
        const uint32_t A = u & kNib, B = (u >> 1) & kNib, C = (u >> 2) & kNib, Dd = (u >> 3) & kNib;
        const uint32_t col = (~(A | B) & kNib) | ((A & ~B) << 1) | ((B & ~A) << 2) | ((A & B) << 3);
        sel[4 * m + 0] = col & ((~(C | Dd) & kNib) * 0xFu);
        sel[4 * m + 1] = col & ((C & ~Dd) * 0xFu);
        sel[4 * m + 2] = col & ((Dd & ~C) * 0xFu);
        sel[4 * m + 3] = col & ((C & Dd) * 0xFu);
    }
    uint4 W = make_uint4(0u, 0u, 0u, 0u);
    if (RANDOM) W = level_words(s, c);
    constexpr int kPhases = DELAYED ? 3 : 1;
#pragma unroll
    for (int ph = 0; ph < kPhases; ++ph) {
        uint32_t cand[16];
        uint32_t pmin = 0u, pmax = 0u;
#pragma unroll
        for (int R = 0; R < 16; ++R) {
            const bool last_row = (R & 3) == 3;
            uint32_t mask = 0xFFFFFFFFu;  // columns of this phase in row R
            if (DELAYED) {
                if (ph == 0) mask = last_row ? 0u : 0x77777777u;
                if (ph == 1) mask = last_row ? 0x77777777u : 0x88888888u;
                if (ph == 2) mask = last_row ? 0x88888888u : 0u;
            }
            const uint32_t x = X[R];
            const uint32_t xr = __funnelshift_r(x, E >> R, 1);
            const uint32_t y = Y[R], yd = (R < 15) ? Y[(R + 1) & 15] : D;
            if (SPEC == 1)
                cand[R] = sel[R] & mask & ~x & xr & ~y & yd;  // the minima
            else
                cand[R] = sel[R] & mask & (x ^ xr) & (y ^ yd) & ~(x ^ y);
        }
        if (RANDOM) {
#pragma unroll
            for (int m = 0; m < 4; ++m) {
                uint32_t mn = 0u, mx = 0u;
#pragma unroll
                for (int r = 0; r < 4; ++r) {
                    mn |= cand[4 * m + r] & ~X[4 * m + r];
                    mx |= cand[4 * m + r] & X[4 * m + r];
                }
                if (SPEC != 2) {
                    mn &= c.p_random;
                    mx &= c.q_random;
                }
                pmin |= ((mn | (mn >> 1) | (mn >> 2) | (mn >> 3)) & kNib) << m;
                pmax |= ((mx | (mx >> 1) | (mx >> 2) | (mx >> 3)) & kNib) << m;
            }
            draws += __popc(pmin | pmax);
        }
        uint32_t acc = 0u;
        if (RANDOM) {
            acc = accept_candidates<kPreDb>(pmin, pmax, W, c, tp);
            net += random_net(acc, pmin, pmax);
        }
        uint32_t dE = 0u, dB0 = 0u, dD = 0u, dY0 = 0u;
#pragma unroll
        for (int R = 0; R < 16; ++R) {
            const int m = R >> 2;
            uint32_t amin = c.p_always, amax = c.q_always;
            if (RANDOM) {
                const uint32_t spread = ((acc >> m) & kNib) * 0xFu;
                amin |= spread & c.p_random;
                amax |= spread & c.q_random;
            }
            const uint32_t x = X[R];
            uint32_t f;
            if (SPEC == 1) {
                f = cand[R];
                net += __popc(f);
            } else if (SPEC == 2) {
                f = cand[R] & ((acc >> m) & kNib) * 0xFu;
            } else {
                f = cand[R] & ((~x & amin) | (x & amax));
                net += always_net<RANDOM>(f, x, c);
            }
            X[R] = x ^ f ^ (f << 1);
            Y[R] ^= f;
            if (R < 15)
                Y[(R + 1) & 15] ^= f;
            else {
                D ^= f;
                dD = f;
            }
            dE |= (f >> 31) << R;
            dB0 |= (f & 1u) << R;
            if (R == 0) dY0 = f;
        }
        // exchange with the neighbouring lanes (all lanes take part)
        E ^= dE;
        const uint32_t vr = __shfl_up_sync(kFull, dE, 1);
        const uint32_t vl = __shfl_down_sync(kFull, dB0, 1);
        if (c.gx > 0) {
#pragma unroll
            for (int r = 0; r < 16; ++r) X[r] ^= (vr >> r) & 1u;
        }
        if (c.gx < c.GX - 1) E ^= vl;
        const uint32_t vd = __shfl_up_sync(kFull, dD, c.GX);
        const uint32_t vu = __shfl_down_sync(kFull, dY0, c.GX);
        if (c.gy > 0) Y[0] ^= vd;
        if (c.gy < c.GY - 1) D ^= vu;
    }
}

// A collective step of DTrDTr (Sec. 4.1.2): DT whose
// block-layer origin moves after every step, the cell grid wrapping around
// the sub-tile.  With the active sub-cell of every cell starting at column c0
// and row R0 (uniform in [0, 4): the set's offset plus the moved origin), the
// attempt of TC (j, m) of a lane is at (4j + c0 + rx, 4m + R0 + ry).  For
// c0 = 3 the pair of TC 7 reaches column 32, i.e. column 0 of the lane to the
// right (of the sub-tile's first lane, for the last lane: the wrap); for
// R0 = 3 the pair of TC row 3 reaches row 16, row 0 of the lane below (or of
// the first lane row), and TC (7, 3) can reach the lane diagonally below.
// The lane holding such a site tests it; the candidate goes back to the
// owning lane, which draws its acceptance with its own level words (so the
// uniforms, and the order of ties, stay those of the owning thread cell), and
// the decision returns to the holder, which flips.  The neighbour copies E, D
// are kept as in DT: the lattice itself does not wrap inside the sub-tile.
// As for DT the step runs in three phases (candidates and flips specialised
// on R0, one copy of the acceptance code between them).
struct DtrLanes {
    int lL, lR, lA, lB, lAL, lBR;  // lanes left, right, above, below, above-left, below-right (wrapping)
};

__device__ __forceinline__ DtrLanes dtr_lanes(const LaneCtx &c) {
    const int gxl = c.gx == 0 ? c.GX - 1 : c.gx - 1, gxr = c.gx == c.GX - 1 ? 0 : c.gx + 1;
    const int gya = c.gy == 0 ? c.GY - 1 : c.gy - 1, gyb = c.gy == c.GY - 1 ? 0 : c.gy + 1;
    DtrLanes n;
    n.lL = gxl + c.gy * c.GX;
    n.lR = gxr + c.gy * c.GX;
    n.lA = c.gx + gya * c.GX;
    n.lB = c.gx + gyb * c.GX;
    n.lAL = gxl + gya * c.GX;
    n.lBR = gxr + gyb * c.GX;
    return n;
}

// v[k] for a run-time k in 0..3 (k uniform over the warp: selects, no branch).
__device__ __forceinline__ uint32_t pick4(uint32_t k, uint32_t v0, uint32_t v1, uint32_t v2, uint32_t v3) {
    const uint32_t lo = (k & 1u) ? v1 : v0, hi = (k & 1u) ? v3 : v2;
    return (k & 2u) ? hi : lo;
}

// Phase 1.  The row phase R0 is a run-time value (one copy of the code for all
// four phases; four specialised copies overflowed the instruction caches).
// ca[m], cb[m]: candidates in rows a = 4m+R0 and b = a+1 held by this lane;
// row 16 (m = 3, R0 = 3) is the lane below's row 0, and cb[3] then holds this
// lane's row 0 (the wrapped row of the lane above) instead.
// pmin / pmax: packed candidates of this lane's own thread cells.
template <bool RANDOM>
__device__ __forceinline__ void dtr_candidates(const uint32_t (&X)[16], const uint32_t (&Y)[16], uint32_t E,
                                               uint32_t D, const uint4 &site, uint32_t s, uint32_t c0,
                                               uint32_t R0, const LaneCtx &c, const DtrLanes &n,
                                               uint32_t (&ca)[4], uint32_t (&cb)[4], uint32_t &pmin,
                                               uint32_t &pmax) {
    const bool SX = c0 == 3u;  // pairs reach column 32 (uniform over the warp)
    const bool SY = R0 == 3u;  // pairs reach row 16
    const uint32_t sw[4] = {site.x, site.y, site.z, site.w};
    const uint32_t par = 2u * (s & 1u);
    // Selected sites: own thread cells in place, those past column 31 in xw
    // (bit = row; bit 16 = row 16), those in row 16 in yw (bit = column).
    uint32_t xw = 0u, yw = 0u;
#pragma unroll
    for (int m = 0; m < 4; ++m) {
        const uint32_t u = sw[m] >> par;
        const uint32_t col = ((u & kNib) << 1) | (~u & kNib);  // bit 4j + rx
        const uint32_t yoff = ((u >> 1) & kNib) * 0xFu;         // thread cells with ry = 1
        const uint64_t a64 = static_cast<uint64_t>(col & ~yoff) << c0;
        const uint64_t b64 = static_cast<uint64_t>(col & yoff) << c0;
        const uint32_t ya = 4u * m + R0;
        ca[m] = static_cast<uint32_t>(a64);
        xw |= static_cast<uint32_t>(a64 >> 32) << ya;
        if (m == 3 && SY) {
            cb[m] = 0u;
            yw = static_cast<uint32_t>(b64);
            xw |= static_cast<uint32_t>(b64 >> 32) << 16;
        } else {
            cb[m] = static_cast<uint32_t>(b64);
            xw |= static_cast<uint32_t>(b64 >> 32) << (ya + 1u);
        }
    }
    // sites of neighbouring lanes' thread cells held by this lane
    if (SX) {
        const uint32_t v = __shfl_sync(kFull, xw, n.lL);
#pragma unroll
        for (int m = 0; m < 4; ++m) {
            const uint32_t ya = 4u * m + R0;
            ca[m] |= (v >> ya) & 1u;
            if (!(m == 3 && SY)) cb[m] |= (v >> (ya + 1u)) & 1u;
        }
    }
    if (SY) {
        const uint32_t v = __shfl_sync(kFull, yw, n.lA);
        const uint32_t corner = SX ? (__shfl_sync(kFull, xw, n.lAL) >> 16) & 1u : 0u;
        cb[3] = v | corner;  // row 0
    }
    // eligibility; rows a and b of TC row m picked by the row phase (for
    // m = 3 the row after 15 is D for Y, and row b = "16" is row 0)
    uint32_t cw = 0u;  // column-0 candidates: minima in bits 0..15, maxima in 16..31 (row = bit)
    uint32_t xa_[4], xb_[4];
#pragma unroll
    for (int m = 0; m < 4; ++m) {
        const int r = 4 * m;
        const uint32_t X4 = m < 3 ? X[(r + 4) & 15] : X[0];
        const uint32_t Y4 = m < 3 ? Y[(r + 4) & 15] : D;
        const uint32_t Yb4 = m < 3 ? Y[(r + 4) & 15] : Y[0];  // row b's own Y when b = "16"
        const uint32_t Y5 = m < 3 ? Y[(r + 5) & 15] : Y[1];
        const uint32_t ya = static_cast<uint32_t>(r) + R0, yb = (ya + 1u) & 15u;
        const uint32_t xa = pick4(R0, X[r], X[r + 1], X[r + 2], X[r + 3]);
        const uint32_t yA = pick4(R0, Y[r], Y[r + 1], Y[r + 2], Y[r + 3]);
        const uint32_t yAd = pick4(R0, Y[r + 1], Y[r + 2], Y[r + 3], Y4);
        const uint32_t xb = pick4(R0, X[r + 1], X[r + 2], X[r + 3], X4);
        const uint32_t yB = pick4(R0, Y[r + 1], Y[r + 2], Y[r + 3], Yb4);
        const uint32_t yBd = pick4(R0, Y[r + 2], Y[r + 3], Y4, Y5);
        ca[m] &= (xa ^ __funnelshift_r(xa, E >> ya, 1)) & (yA ^ yAd) & ~(xa ^ yA);
        cb[m] &= (xb ^ __funnelshift_r(xb, E >> yb, 1)) & (yB ^ yBd) & ~(xb ^ yB);
        xa_[m] = xa;
        xb_[m] = xb;
        if (RANDOM) {
            cw |= ((ca[m] & ~xa & 1u) << ya) | ((ca[m] & xa & 1u) << (ya + 16u));
            cw |= ((cb[m] & ~xb & 1u) << yb) | ((cb[m] & xb & 1u) << (yb + 16u));
        }
    }
    pmin = 0u;
    pmax = 0u;
    if (RANDOM) {
        const uint32_t cwR = SX ? __shfl_sync(kFull, cw, n.lR) : 0u;
        const uint32_t cwBR = (SX && SY) ? __shfl_sync(kFull, cw, n.lBR) : 0u;
        uint32_t bmin = 0u, bmax = 0u;  // row 0 of the lane below
        if (SY) {
            bmin = __shfl_sync(kFull, cb[3] & ~X[0], n.lB);
            bmax = __shfl_sync(kFull, cb[3] & X[0], n.lB);
        }
#pragma unroll
        for (int m = 0; m < 4; ++m) {
            const uint32_t ya = 4u * m + R0, yb = ya + 1u;
            uint32_t mnl = ca[m] & ~xa_[m], mxl = ca[m] & xa_[m];
            uint32_t mnh = (cwR >> ya) & 1u, mxh = (cwR >> (ya + 16u)) & 1u;
            if (m == 3 && SY) {
                mnl |= bmin;
                mxl |= bmax;
                mnh |= cwBR & 1u;
                mxh |= (cwBR >> 16) & 1u;
            } else {
                mnl |= cb[m] & ~xb_[m];
                mxl |= cb[m] & xb_[m];
                mnh |= (cwR >> yb) & 1u;
                mxh |= (cwR >> (yb + 16u)) & 1u;
            }
            // align each cell's pair to bits 4j, 4j+1, then pack to bit 4j+m
            const uint32_t cmn = __funnelshift_r(mnl, mnh, c0) & c.p_random;
            const uint32_t cmx = __funnelshift_r(mxl, mxh, c0) & c.q_random;
            pmin |= ((cmn | (cmn >> 1)) & kNib) << m;
            pmax |= ((cmx | (cmx >> 1)) & kNib) << m;
        }
        // A lane outside the sub-tile can read a sub-tile lane's candidates
        // through the wrapped lane indices; it owns no thread cell.
        if (!c.active) {
            pmin = 0u;
            pmax = 0u;
        }
    }
}

// Phase 3: flips of the accepted candidates (acc: this lane's packed
// acceptance bits), then the exchange of the neighbour copies.  The flips of
// row r come from TC row m = r / 4 when r % 4 is R0 (row a) or R0 + 1 (row b),
// and from TC row m - 1 (mod 4: row 0 takes the wrapped row of TC row 3) when
// r % 4 = 0 and R0 = 3.
template <bool RANDOM>
__device__ __forceinline__ void dtr_apply(uint32_t (&X)[16], uint32_t (&Y)[16], uint32_t &E, uint32_t &D,
                                          uint32_t c0, uint32_t R0, uint32_t acc, const uint32_t (&ca)[4],
                                          const uint32_t (&cb)[4], const LaneCtx &c, const DtrLanes &n,
                                          int &net) {
    const bool SX = c0 == 3u;
    const bool SY = R0 == 3u;
    uint32_t accL = 0u, accA = 0u, accAL = 0u;
    if (RANDOM) {
        if (SX) accL = __shfl_sync(kFull, acc, n.lL);
        if (SY) accA = __shfl_sync(kFull, acc, n.lA);
        if (SX && SY) accAL = __shfl_sync(kFull, acc, n.lAL);
    }
    // accepted candidates of rows a and b of every TC row (fb[3] with R0 = 3: row 0)
    uint32_t fa[4], fb[4];
#pragma unroll
    for (int m = 0; m < 4; ++m) {
        const int r = 4 * m;
        const uint32_t xa = pick4(R0, X[r], X[r + 1], X[r + 2], X[r + 3]);
        const uint32_t xb = pick4(R0, X[r + 1], X[r + 2], X[r + 3], m < 3 ? X[(r + 4) & 15] : X[0]);
        uint32_t amin = c.p_always, amax = c.q_always, bmin = c.p_always, bmax = c.q_always;
        if (RANDOM) {
            const uint32_t own = ((acc >> m) & kNib) * 0xFu;
            const uint32_t left = ((accL >> m) & kNib) * 0xFu;
            const uint32_t cols = __funnelshift_l(left, own, c0);
            // row 0 with R0 = 3: thread cells of the lanes above
            const uint32_t cols0 = __funnelshift_l(((accAL >> 3) & kNib) * 0xFu, ((accA >> 3) & kNib) * 0xFu, c0);
            const uint32_t colb = (m == 3 && SY) ? cols0 : cols;
            amin |= cols & c.p_random;
            amax |= cols & c.q_random;
            bmin |= colb & c.p_random;
            bmax |= colb & c.q_random;
        }
        fa[m] = ca[m] & ((~xa & amin) | (xa & amax));
        fb[m] = cb[m] & ((~xb & bmin) | (xb & bmax));
        net += always_net<RANDOM>(fa[m], xa, c) + always_net<RANDOM>(fb[m], xb, c);
    }
    uint32_t dE = 0u, dB0 = 0u, F_prev = 0u;
#pragma unroll
    for (int r = 0; r < 16; ++r) {
        const int m = r >> 2;
        const uint32_t k = static_cast<uint32_t>(r & 3);
        uint32_t F = (R0 == k ? fa[m] : 0u) | (R0 + 1u == k ? fb[m] : 0u);
        if (k == 0u && SY) F |= fb[(m + 3) & 3];
        X[r] ^= F * 3u;      // F ^ (F << 1): the row's flips are at least three columns apart
        Y[r] ^= F ^ F_prev;  // its own Y, and Y(s+y) of the row above
        dE |= (F >> 31) << r;
        dB0 |= (F & 1u) << r;
        F_prev = F;
    }
    D ^= F_prev;  // Y(s+y) of row 15
    const uint32_t dD = F_prev;
    const uint32_t dY0 = (R0 == 0u ? fa[0] : 0u) | (SY ? fb[3] : 0u);  // the flips of row 0
    E ^= dE;
    const uint32_t vr = __shfl_up_sync(kFull, dE, 1);
    const uint32_t vl = __shfl_down_sync(kFull, dB0, 1);
    if (c.gx > 0) {
#pragma unroll
        for (int r = 0; r < 16; ++r) X[r] ^= (vr >> r) & 1u;
    }
    if (c.gx < c.GX - 1) E ^= vl;
    const uint32_t vd = __shfl_up_sync(kFull, dD, c.GX);
    const uint32_t vu = __shfl_down_sync(kFull, dY0, c.GX);
    if (c.gy > 0) Y[0] ^= vd;
    if (c.gy < c.GY - 1) D ^= vu;
}

// Where a lane's group lies in the planar lattice: the two words wA, wB of
// every row that hold its 32 sites (from bit sh of wA), its first row ybase
// and the sub-tile's halo row yh.
struct LaneGeom {
    uint32_t *Xp, *Yp;
    uint32_t sh, wA, wB, ybase, yh;
};

// (y0 in buffer rows; the Y plane follows plane_rows rows of X.)
__device__ __forceinline__ LaneGeom lane_geom(uint32_t *lat, uint32_t L, uint32_t plane_rows, uint32_t wpr,
                                              uint32_t By, uint32_t x0, uint32_t y0, const LaneCtx &c) {
    LaneGeom q;
    q.Xp = lat;
    q.Yp = lat + static_cast<size_t>(plane_rows) * wpr;
    q.sh = x0 & 31u;
    q.wA = ((x0 >> 5) + static_cast<uint32_t>(c.gx)) % wpr;
    q.wB = (q.wA + 1u == wpr) ? 0u : q.wA + 1u;
    q.ybase = y0 + 16u * static_cast<uint32_t>(c.gy);
    if (q.ybase >= L) q.ybase -= L;
    q.yh = y0 + By;
    if (q.yh >= L) q.yh -= L;
    return q;
}

// Stage the lane's group: 16 rows of X and Y, funnel-shifted to local bit 0;
// E: column 0 of the right neighbour (the halo column x0 + Bx for the last
// lane column); D: row 0 of the lane below (the halo row y0 + By for the last
// lane row).
__device__ __forceinline__ void stage_lane(const LaneGeom &q, uint32_t L, uint32_t wpr, uint32_t Bx, uint32_t x0,
                                           bool active, const LaneCtx &c, uint32_t (&X)[16], uint32_t (&Y)[16],
                                           uint32_t &E, uint32_t &D) {
    const uint32_t *const Xp = q.Xp;
    const uint32_t *const Yp = q.Yp;
#pragma unroll
    for (int r = 0; r < 16; ++r) {
        X[r] = 0u;
        Y[r] = 0u;
    }
    if (active) {
#pragma unroll
        for (int r = 0; r < 16; ++r) {
            uint32_t yr = q.ybase + r;
            if (yr >= L) yr -= L;
            const size_t ro = static_cast<size_t>(yr) * wpr;
            X[r] = __funnelshift_r(Xp[ro + q.wA], Xp[ro + q.wB], q.sh);
            Y[r] = __funnelshift_r(Yp[ro + q.wA], Yp[ro + q.wB], q.sh);
        }
    }
    uint32_t b0 = 0;
#pragma unroll
    for (int r = 0; r < 16; ++r) b0 |= (X[r] & 1u) << r;
    E = __shfl_down_sync(kFull, b0, 1);
    D = __shfl_down_sync(kFull, Y[0], c.GX);
    if (active && c.gx == c.GX - 1) {  // halo column x0 + Bx
        uint32_t xc = x0 + Bx;
        if (xc >= L) xc -= L;
        const uint32_t wc = xc >> 5, bc = xc & 31u;
        E = 0u;
#pragma unroll
        for (int r = 0; r < 16; ++r) {
            uint32_t yr = q.ybase + r;
            if (yr >= L) yr -= L;
            E |= ((Xp[static_cast<size_t>(yr) * wpr + wc] >> bc) & 1u) << r;
        }
    }
    if (active && c.gy == c.GY - 1) {  // halo row y0 + By
        const size_t ro = static_cast<size_t>(q.yh) * wpr;
        D = __funnelshift_r(Yp[ro + q.wA], Yp[ro + q.wB], q.sh);
    }
}

template <bool LANE_SETS>
__device__ __forceinline__ void write_back(const LaneGeom &q, uint32_t L, uint32_t wpr, bool active,
                                           const LaneCtx &c, const uint32_t (&X)[16], const uint32_t (&Y)[16],
                                           uint32_t E, uint32_t D) {
    uint32_t *const Xp = q.Xp;
    uint32_t *const Yp = q.Yp;
    const uint32_t sh = q.sh, wA = q.wA, wB = q.wB, ybase = q.ybase, yh = q.yh;
    // Write back.  Global word wA of a row receives the high bits of the left
    // lane and the low bits of this lane; the leftmost lane shares word wA
    // with the bits left of x0, the rightmost lane also owns the low bits of
    // word wB (its own high bits, and for X the halo-column bit).  The bits of
    // those shared words outside the sub-tile belong to neighbouring sub-tiles,
    // which this device step does not update, and no other warp writes these
    // words (active sub-tiles are at least 32 sites apart).  Full words are
    // stored.  Shared words are merged in one of two ways:
    //  * a warp holding one sub-tile (few shared words per lane): an AND/OR
    //    reduction pair, which returns nothing, so the warp does not wait;
    //  * a warp holding several small sub-tiles (many shared words per lane):
    //    a fresh read of the outside bits, all reads of eight rows before
    //    their stores (one wait for memory per eight rows), and one plain
    //    store per word; there the reductions' throughput would bind the step.
    const bool left_edge = active && c.gx == 0 && sh != 0u;
    const bool right_edge = active && c.gx == c.GX - 1;
    const uint32_t lo_mask = (1u << sh) - 1u;  // bits [0, sh): left of x0 in word wA
    const uint32_t xb_mask = (2u << sh) - 1u;  // bits [0, sh]: ours in word wB of X (halo bit at sh)
    const bool by_read = LANE_SETS;
#pragma unroll
    for (int h = 0; h < 16; h += 8) {
        uint32_t oX[8], oY[8];  // outside bits of the lane's edge words (wA's in lo_mask, wB's above)
        if (by_read) {
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                uint32_t yr = ybase + h + i;
                if (yr >= L) yr -= L;
                const size_t ro = static_cast<size_t>(yr) * wpr;
                oX[i] = 0u;
                oY[i] = 0u;
                if (left_edge) {
                    oX[i] = Xp[ro + wA] & lo_mask;
                    oY[i] = Yp[ro + wA] & lo_mask;
                }
                if (right_edge) {
                    oX[i] |= Xp[ro + wB] & ~xb_mask;
                    oY[i] |= Yp[ro + wB] & ~lo_mask;
                }
            }
        }
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int r = h + i;
            const uint32_t leftX = __shfl_up_sync(kFull, X[r], 1);
            const uint32_t leftY = __shfl_up_sync(kFull, Y[r], 1);
            if (active) {
                uint32_t yr = ybase + r;
                if (yr >= L) yr -= L;
                const size_t ro = static_cast<size_t>(yr) * wpr;
                if (left_edge) {
                    if (by_read) {
                        Xp[ro + wA] = (oX[i] & lo_mask) | (X[r] << sh);
                        Yp[ro + wA] = (oY[i] & lo_mask) | (Y[r] << sh);
                    } else {
                        reduce_bits(&Xp[ro + wA], X[r] << sh, ~lo_mask);
                        reduce_bits(&Yp[ro + wA], Y[r] << sh, ~lo_mask);
                    }
                } else {
                    Xp[ro + wA] = __funnelshift_l(leftX, X[r], sh);
                    Yp[ro + wA] = __funnelshift_l(leftY, Y[r], sh);
                }
                if (right_edge) {
                    const uint32_t hiX = (sh ? (X[r] >> (32u - sh)) : 0u) | (((E >> r) & 1u) << sh);
                    const uint32_t hiY = sh ? (Y[r] >> (32u - sh)) : 0u;
                    if (by_read) {
                        Xp[ro + wB] = (oX[i] & ~xb_mask) | hiX;
                        if (sh) Yp[ro + wB] = (oY[i] & ~lo_mask) | hiY;
                    } else {
                        reduce_bits(&Xp[ro + wB], hiX, xb_mask);
                        if (sh) reduce_bits(&Yp[ro + wB], hiY, lo_mask);
                    }
                }
            }
        }
    }
    {
        const bool d_row = active && c.gy == c.GY - 1;
        const size_t ro = static_cast<size_t>(yh) * wpr;
        uint32_t oD = 0u;
        if (by_read && d_row) {
            if (left_edge) oD = Yp[ro + wA] & lo_mask;
            if (right_edge && sh) oD |= Yp[ro + wB] & ~lo_mask;
        }
        const uint32_t leftD = __shfl_up_sync(kFull, D, 1);
        if (d_row) {
            if (left_edge) {
                if (by_read)
                    Yp[ro + wA] = (oD & lo_mask) | (D << sh);
                else
                    reduce_bits(&Yp[ro + wA], D << sh, ~lo_mask);
            } else {
                Yp[ro + wA] = __funnelshift_l(leftD, D, sh);
            }
            if (right_edge && sh) {
                if (by_read)
                    Yp[ro + wB] = (oD & ~lo_mask) | (D >> (32u - sh));
                else
                    reduce_bits(&Yp[ro + wB], D >> (32u - sh), lo_mask);
            }
        }
    }
}

// Device step on one sub-tile (Bx x By sites at (x0, y0)) held by the lanes of
// one warp that share it: stage the lane's group from the planar lattice,
// run the 16 single-hit collective steps, write back.  LANE_SETS: lanes of the
// warp may belong to different sub-tiles (each with its own set draws).
// SCHEME: 0 DTrDT, 1 DTrDB with all attempts of a step together, 2 DTrDB with
// delayed borders, 3 DTrDTr, 4 DTrDT with deposition only (p = 1, q = 0),
// 5 DTrDT with both rates strictly inside (0, 1), 6 DTrDB with deposition only,
// 7 DTrDB with delayed borders and both rates random.
template <bool RANDOM, bool LANE_SETS, int SCHEME = 0>
__device__ __forceinline__ void run_subtile(uint32_t *lat, uint32_t L, uint32_t plane_rows, uint32_t wpr,
                                            uint32_t Bx, uint32_t By, uint32_t x0, uint32_t y0, bool active,
                                            const LaneCtx &c, uint32_t *ring, int &net, int &draws,
                                            int &tails) {
    TailPool tp;
    tp.ring = ring + static_cast<uint32_t>(kRingWordsPerLane) * c.g;  // the lane's own slot
    tp.head = 0u;
    tp.end = 0u;
    tp.rounds = 0u;
    const LaneGeom q = lane_geom(lat, L, plane_rows, wpr, By, x0, y0, c);
    uint32_t X[16], Y[16], E, D;
    stage_lane(q, L, wpr, Bx, x0, active, c, X, Y, E, D);

    // Block layer: 16 single-hit collective steps.
    const uint4 setw = philox4x32_10(c.t, c.k, c.T, kTagSet << 28, c.k0, c.k1);
    uint4 site = make_uint4(0u, 0u, 0u, 0u);
    uint4 borg = make_uint4(0u, 0u, 0u, 0u);
    if (SCHEME == 3) borg = philox4x32_10(c.t, c.k, c.T, kTagBorg << 28, c.k0, c.k1);
    for (uint32_t s = 0; s < 16u; ++s) {
        if (SCHEME == 3) {
            // DTrDTr: the set, plus a block-layer origin (ax, ay) per step
            if ((s & 1u) == 0u)
                site = philox4x32_10(c.t, c.k | ((s >> 1) << 2), c.T, (kTagSite << 28) | c.g, c.k0, c.k1);
            const uint32_t d = (setw.x >> (2u * s)) & 3u;
            const uint32_t bw = (s < 4u) ? borg.x : (s < 8u) ? borg.y : (s < 12u) ? borg.z : borg.w;
            const uint32_t byte = (bw >> (8u * (s & 3u))) & 0xFFu;
            const uint32_t c0 = ((byte & 3u) + 2u * (d & 1u)) & 3u;
            const uint32_t r0 = (((byte >> 4) & 3u) + 2u * (d >> 1)) & 3u;
            const DtrLanes n = dtr_lanes(c);
            uint32_t ca[4], cb[4], pmin, pmax;
            dtr_candidates<RANDOM>(X, Y, E, D, site, s, c0, r0, c, n, ca, cb, pmin, pmax);
            uint32_t acc = 0u;
            if (RANDOM) {
                draws += __popc(pmin | pmax);
                acc = accept_candidates<SCHEME == 3 ? kPreDtr : (LANE_SETS ? kPrePacked : kPreDt)>(pmin, pmax, level_words(s, c), c, tp);
                net += random_net(acc, pmin, pmax);
            }
            dtr_apply<RANDOM>(X, Y, E, D, c0, r0, acc, ca, cb, c, n, net);
            continue;
        }
        if (SCHEME == 1 || SCHEME == 2 || SCHEME == 6 || SCHEME == 7) {
            // DB: one site word per TC row and step, 4 bits per cell
            site = philox4x32_10(c.t, c.k | (s << 2), c.T, (kTagSiteDb << 28) | c.g, c.k0, c.k1);
            if (SCHEME == 2)
                db_step<RANDOM, true>(X, Y, E, D, site, s, c, tp, net, draws);
            else if (SCHEME == 7)
                db_step<RANDOM, true, 2>(X, Y, E, D, site, s, c, tp, net, draws);
            else if (SCHEME == 6)
                db_step<RANDOM, false, 1>(X, Y, E, D, site, s, c, tp, net, draws);
            else
                db_step<RANDOM, false>(X, Y, E, D, site, s, c, tp, net, draws);
            continue;
        }
        if ((s & 1u) == 0u)
            site = philox4x32_10(c.t, c.k | ((s >> 1) << 2), c.T, (kTagSite << 28) | c.g, c.k0, c.k1);
        else
            site = make_uint4(site.x >> 2, site.y >> 2, site.z >> 2, site.w >> 2);
        // the set (every lane of a one-sub-tile warp drew the same one; the broadcast
        // from lane 0 lets the compiler treat the branches on it as warp-uniform)
        const uint32_t d_own = (setw.x >> (2u * s)) & 3u;
        const uint32_t d = LANE_SETS ? d_own : __shfl_sync(kFull, d_own, 0);
        uint32_t cnd0[4], cnd1[4], pmin, pmax;
        constexpr int kSpec = SCHEME == 4 ? 1 : SCHEME == 5 ? 2 : 0;
        if (LANE_SETS)
            step_candidates_rt<RANDOM, kSpec>(X, Y, E, D, site, s, d & 1u, d >> 1, c, cnd0, cnd1, pmin, pmax);
        // the candidate phase with the set's column offset as a constant as well
        // (the flip phase stays specialised on the row offset alone: four copies
        // of it measured slower, from instruction-cache pressure)
        else if (d == 3u)
            step_candidates<1, RANDOM, kSpec>(X, Y, E, D, site, s, 1u, c, cnd0, cnd1, pmin, pmax);
        else if (d == 2u)
            step_candidates<1, RANDOM, kSpec>(X, Y, E, D, site, s, 0u, c, cnd0, cnd1, pmin, pmax);
        else if (d == 1u)
            step_candidates<0, RANDOM, kSpec>(X, Y, E, D, site, s, 1u, c, cnd0, cnd1, pmin, pmax);
        else
            step_candidates<0, RANDOM, kSpec>(X, Y, E, D, site, s, 0u, c, cnd0, cnd1, pmin, pmax);
        uint32_t acc = 0u;
        if (RANDOM) {
            draws += __popc(pmin | pmax);
            acc = accept_candidates<SCHEME == 3 ? kPreDtr : (LANE_SETS ? kPrePacked : kPreDt)>(pmin, pmax, level_words(s, c), c, tp);
            net += random_net(acc, pmin, pmax);
        }
        if (LANE_SETS)
            step_apply_rt<RANDOM, kSpec>(X, Y, E, D, d >> 1, acc, cnd0, cnd1, c, net);
        else if (d & 2u)
            step_apply<1, RANDOM, kSpec>(X, Y, E, D, d & 1u, acc, cnd0, cnd1, c, net);
        else
            step_apply<0, RANDOM, kSpec>(X, Y, E, D, d & 1u, acc, cnd0, cnd1, c, net);
    }

    write_back<LANE_SETS>(q, L, wpr, active, c, X, Y, E, D);
    tails = static_cast<int>(tp.rounds);
}

}  // namespace oct
