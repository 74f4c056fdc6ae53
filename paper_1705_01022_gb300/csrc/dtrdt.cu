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
// draws for 0 < p, q < 1 compare all 32 TCs of a lane against P32 at once,
// one random bit level at a time, most significant bit first.
//
// Random streams (Philox-4x32-10, key = seed):
//   MCS draw  (t, 0, 0, MCS<<28): ox, oy, set permutation
//   set draw  (t, k, T, SET<<28): 2 bits per collective step
//   site draw (t, k|(s/2)<<2, T, SITE<<28|g): word m = TC row, bits 4j+2(s&1)
//             (x offset) and 4j+2(s&1)+1 (y offset) for the TC in column j
//   acceptance level words (t, k|(s*8+lb)<<2, T, ACC<<28|g): level l = 4lb+i,
//             bit 4j+m is bit 31-l of the uniform of TC (j, m)
#include "oct_internal.h"
#include "philox.cuh"

namespace oct {
namespace {

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
__device__ __forceinline__ void merge_bits(uint32_t *w, uint32_t v, uint32_t mask) {
    if (mask == 0xFFFFFFFFu) {
        *w = v;
        return;
    }
    atomicAnd(w, v | ~mask);
    atomicOr(w, v & mask);
}

struct LaneCtx {
    uint32_t t, k, T, g;
    uint32_t k0, k1;
    uint32_t thr_p, thr_q;
    uint32_t p_always, q_always, p_random, q_random;
    int gx, gy, GX, GY;
};

// Acceptance of the packed candidates (bit 4j+m = thread cell column j, TC
// row m): u < P32 is decided at the first random level bit that differs from
// P32's bit, most significant first; all 32 thread cells of the lane advance
// together, four levels per Philox block.
__device__ __forceinline__ uint32_t accept_levels(uint32_t pmin, uint32_t pmax, uint32_t s,
                                                  const LaneCtx &c) {
    uint32_t acc = 0, und = pmin | pmax;
    for (uint32_t lb = 0; lb < 8u && und != 0u; ++lb) {
        const uint4 W = philox4x32_10(c.t, c.k | ((s * 8u + lb) << 2), c.T, (kTagAcc << 28) | c.g,
                                      c.k0, c.k1);
        const uint32_t lw[4] = {W.x, W.y, W.z, W.w};
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const uint32_t bit = 31u - (4u * lb + i);
            const uint32_t tb = (((c.thr_p >> bit) & 1u) ? pmin : 0u) | (((c.thr_q >> bit) & 1u) ? pmax : 0u);
            acc |= und & tb & ~lw[i];
            und &= ~(tb ^ lw[i]);
        }
    }
    return acc;
}

// One collective step with sub-cell set (dx, DY).  X/Y hold the lane's 16
// rows, E bit r the X bit just right of row r, D the Y row just below row 15.
// An attempt at s is eligible iff X(s) != X(s+x), Y(s) != Y(s+y) and
// X(s) == Y(s): then X(s) = 0 is the minimum of Eq. (1), X(s) = 1 the maximum.
template <int DY, bool RANDOM>
__device__ __forceinline__ void collective_step(uint32_t (&X)[16], uint32_t (&Y)[16], uint32_t &E,
                                                uint32_t &D, const uint4 &site, uint32_t s,
                                                uint32_t dx, const LaneCtx &c, int &net, int &draws) {
    const uint32_t sw[4] = {site.x, site.y, site.z, site.w};
    const uint32_t par = 2u * (s & 1u);
    const uint32_t sh2 = 2u * dx;
    uint32_t cnd0[4], cnd1[4];
#pragma unroll
    for (int m = 0; m < 4; ++m) {
        // Site draw: bit 4j = x offset, bit 4j+1 = y offset of TC column j.
        const uint32_t u = sw[m] >> par;
        const uint32_t col = (((u & kNib) << 1) | (~u & kNib)) << sh2;
        const uint32_t yoff = ((u >> 1) & kNib) * 0xFu;
        const int r0 = 4 * m + 2 * DY, r1 = r0 + 1;
        const uint32_t xa = X[r0], xb = X[r1];
        const uint32_t xra = __funnelshift_r(xa, E >> r0, 1);
        const uint32_t xrb = __funnelshift_r(xb, E >> r1, 1);
        const uint32_t ya = Y[r0], yb = Y[r1];
        const uint32_t yc = (r1 + 1 < 16) ? Y[(r1 + 1) & 15] : D;
        cnd0[m] = col & ~yoff & (xa ^ xra) & (ya ^ yb) & ~(xa ^ ya);
        cnd1[m] = col & yoff & (xb ^ xrb) & (yb ^ yc) & ~(xb ^ yb);
    }

    uint32_t acc = 0;
    if (RANDOM) {
        uint32_t pmin = 0, pmax = 0;
#pragma unroll
        for (int m = 0; m < 4; ++m) {
            const int r0 = 4 * m + 2 * DY, r1 = r0 + 1;
            const uint32_t mn = (cnd0[m] & ~X[r0]) | (cnd1[m] & ~X[r1]);
            const uint32_t mx = (cnd0[m] & X[r0]) | (cnd1[m] & X[r1]);
            const uint32_t cmn = mn & c.p_random, cmx = mx & c.q_random;
            pmin |= (((cmn >> sh2) | (cmn >> (sh2 + 1u))) & kNib) << m;
            pmax |= (((cmx >> sh2) | (cmx >> (sh2 + 1u))) & kNib) << m;
        }
        draws += __popc(pmin | pmax);
        acc = accept_levels(pmin, pmax, s, c);
    }

    uint32_t f0s[4], f1s[4];
#pragma unroll
    for (int m = 0; m < 4; ++m) {
        const int r0 = 4 * m + 2 * DY, r1 = r0 + 1;
        uint32_t amin = c.p_always, amax = c.q_always;
        if (RANDOM) {
            const uint32_t spread = ((acc >> m) & kNib) * 0xFu;
            amin |= spread & c.p_random;
            amax |= spread & c.q_random;
        }
        const uint32_t xa = X[r0], xb = X[r1];
        // accepted minima are where the candidate has X(s) = 0
        const uint32_t f0 = cnd0[m] & ((~xa & amin) | (xa & amax));
        const uint32_t f1 = cnd1[m] & ((~xb & amin) | (xb & amax));
        net += __popc((f0 & ~xa) | (f1 & ~xb)) - __popc((f0 & xa) | (f1 & xb));
        X[r0] = xa ^ f0 ^ (f0 << 1);
        X[r1] = xb ^ f1 ^ (f1 << 1);
        Y[r0] ^= f0;
        Y[r1] ^= f0 ^ f1;
        if (r1 + 1 < 16)
            Y[(r1 + 1) & 15] ^= f1;
        else
            D ^= f1;
        f0s[m] = f0;
        f1s[m] = f1;
    }

    // Keep the neighbour copies consistent.
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

template <bool RANDOM>
__global__ void __launch_bounds__(kStepWarpsPerBlock * 32, kStepBlocksPerSM)
    dtrdt_step_kernel(const StepArgs a) {
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
    uint32_t *const Xp = a.lat;
    uint32_t *const Yp = a.lat + static_cast<size_t>(L) * wpr;
    const uint32_t sh = x0 & 31u;
    const uint32_t wA = ((x0 >> 5) + static_cast<uint32_t>(c.gx)) % wpr;
    const uint32_t wB = (wA + 1u == wpr) ? 0u : wA + 1u;
    uint32_t ybase = y0 + 16u * static_cast<uint32_t>(c.gy);
    if (ybase >= L) ybase -= L;

    // Stage the group: 16 rows of X and Y, funnel-shifted to local bit 0.
    uint32_t X[16], Y[16];
#pragma unroll
    for (int r = 0; r < 16; ++r) {
        X[r] = 0u;
        Y[r] = 0u;
    }
    if (active) {
#pragma unroll
        for (int r = 0; r < 16; ++r) {
            uint32_t yr = ybase + r;
            if (yr >= L) yr -= L;
            const size_t ro = static_cast<size_t>(yr) * wpr;
            X[r] = __funnelshift_r(Xp[ro + wA], Xp[ro + wB], sh);
            Y[r] = __funnelshift_r(Yp[ro + wA], Yp[ro + wB], sh);
        }
    }
    // E: column 0 of the right neighbour; D: row 0 of the lane below.
    uint32_t b0 = 0;
#pragma unroll
    for (int r = 0; r < 16; ++r) b0 |= (X[r] & 1u) << r;
    uint32_t E = __shfl_down_sync(kFull, b0, 1);
    uint32_t D = __shfl_down_sync(kFull, Y[0], c.GX);
    if (active && c.gx == c.GX - 1) {  // halo column x0 + Bx
        uint32_t xc = x0 + a.Bx;
        if (xc >= L) xc -= L;
        const uint32_t wc = xc >> 5, bc = xc & 31u;
        E = 0u;
#pragma unroll
        for (int r = 0; r < 16; ++r) {
            uint32_t yr = ybase + r;
            if (yr >= L) yr -= L;
            E |= ((Xp[static_cast<size_t>(yr) * wpr + wc] >> bc) & 1u) << r;
        }
    }
    uint32_t yh = y0 + a.By;
    if (yh >= L) yh -= L;
    if (active && c.gy == c.GY - 1) {  // halo row y0 + By
        const size_t ro = static_cast<size_t>(yh) * wpr;
        D = __funnelshift_r(Yp[ro + wA], Yp[ro + wB], sh);
    }

    // Block layer: 16 single-hit collective steps.
    const uint4 setw = philox4x32_10(t, a.k, T, kTagSet << 28, a.k0, a.k1);
    int net = 0, draws = 0;
    uint4 site = make_uint4(0u, 0u, 0u, 0u);
    for (uint32_t s = 0; s < 16u; ++s) {
        if ((s & 1u) == 0u)
            site = philox4x32_10(t, a.k | ((s >> 1) << 2), T, (kTagSite << 28) | c.g, a.k0, a.k1);
        const uint32_t d = (setw.x >> (2u * s)) & 3u;
        if (d & 2u)
            collective_step<1, RANDOM>(X, Y, E, D, site, s, d & 1u, c, net, draws);
        else
            collective_step<0, RANDOM>(X, Y, E, D, site, s, d & 1u, c, net, draws);
    }

    // Write back.  Global word wA of a row receives the high bits of the left
    // lane and the low bits of this lane; the leftmost lane shares word wA
    // with the bits left of x0, the rightmost lane also owns the low bits of
    // word wB (its own high bits, and for X the halo-column bit).  Words shared
    // with sites outside the sub-tile are merged with an AND/OR reduction pair
    // (no read, so no load latency), full words are stored.  No other warp of
    // this device step touches these words: active sub-tiles are at least 32
    // sites apart.
#pragma unroll
    for (int r = 0; r < 16; ++r) {
        const uint32_t leftX = __shfl_up_sync(kFull, X[r], 1);
        const uint32_t leftY = __shfl_up_sync(kFull, Y[r], 1);
        if (active) {
            uint32_t yr = ybase + r;
            if (yr >= L) yr -= L;
            const size_t ro = static_cast<size_t>(yr) * wpr;
            if (c.gx == 0 && sh) {
                merge_bits(&Xp[ro + wA], X[r] << sh, ~0u << sh);
                merge_bits(&Yp[ro + wA], Y[r] << sh, ~0u << sh);
            } else {
                Xp[ro + wA] = __funnelshift_l(leftX, X[r], sh);
                Yp[ro + wA] = __funnelshift_l(leftY, Y[r], sh);
            }
            if (c.gx == c.GX - 1) {
                const uint32_t hiX = sh ? (X[r] >> (32u - sh)) : 0u;
                merge_bits(&Xp[ro + wB], hiX | (((E >> r) & 1u) << sh), (2u << sh) - 1u);
                if (sh) merge_bits(&Yp[ro + wB], Y[r] >> (32u - sh), (1u << sh) - 1u);
            }
        }
    }
    {
        const uint32_t leftD = __shfl_up_sync(kFull, D, 1);
        if (active && c.gy == c.GY - 1) {
            const size_t ro = static_cast<size_t>(yh) * wpr;
            if (c.gx == 0 && sh)
                merge_bits(&Yp[ro + wA], D << sh, ~0u << sh);
            else
                Yp[ro + wA] = __funnelshift_l(leftD, D, sh);
            if (c.gx == c.GX - 1 && sh) merge_bits(&Yp[ro + wB], D >> (32u - sh), (1u << sh) - 1u);
        }
    }

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
    if (any_random)
        dtrdt_step_kernel<true><<<blocks, kStepWarpsPerBlock * 32, 0, st>>>(a);
    else
        dtrdt_step_kernel<false><<<blocks, kStepWarpsPerBlock * 32, 0, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_advance_t(uint32_t *t_ptr, cudaStream_t st) {
    advance_t_kernel<<<1, 1, 0, st>>>(t_ptr);
    return cudaGetLastError();
}

}  // namespace oct
