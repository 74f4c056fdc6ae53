// Internal declarations shared by the library's translation units (host side).
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <string>

#include "oct.h"

namespace oct {

// Arguments of one device-step launch (one set of sub-tiles of one MCS).
struct StepArgs {
    uint32_t *lat;             // planar lattice: X plane, then Y plane
    uint32_t L;                // lateral size
    uint32_t wpr;              // words per row, L / 32
    uint32_t Bx, By;           // sub-tile size in sites
    uint32_t GX, GY;           // groups per sub-tile: Bx / 32 columns, By / 16 rows
    uint32_t tiles_x, tiles_y; // device tiles per direction: L / (2Bx), L / (2By)
    uint32_t k0, k1;           // Philox key
    uint32_t thr_p, thr_q;     // P32(p), P32(q) when the probability is strictly inside (0,1)
    uint32_t p_always, q_always;   // all-ones if p == 1 (resp. q == 1), else 0
    uint32_t p_random, q_random;   // all-ones if 0 < p < 1 (resp. q), else 0
    const uint32_t *t_ptr;     // device-resident MCS counter
    uint32_t k;                // device step 0..3
    unsigned long long *net;   // kNetSlots signed flip counters (two's complement)
    unsigned long long *draws; // kNetSlots counters of attempts that needed an acceptance draw
    unsigned long long *tails; // kNetSlots counters of tail-stream Philox blocks generated
    uint32_t scheme;           // 0: DT; 1: DB (borders together); 2: DB with delayed borders; 3: DTrDTr
    uint32_t cx, cy;           // thread cell in sites (4 x 4, or a coarser DTrDT cell of cells.cu)
    // Row strip of the multi-GPU partition (strip_tiles_y = 0: the whole lattice).
    uint32_t row0;             // global row of buffer row 0
    uint32_t plane_rows;       // rows per bit plane in the buffer (L for the whole lattice)
    uint32_t strip_tiles_y;    // device-tile rows the strip owns (0: all)
};

constexpr int kNetSlots = 1024;
constexpr int kStepWarpsPerBlock = 4;
constexpr int kStepBlocksPerSM = 5;  // occupancy target: 20 warps per SM
constexpr int kStepBlocksPerSMPacked = 4;  // several sub-tiles per warp: per-lane row offsets need more registers

// Launches one device step; returns the CUDA launch status.
cudaError_t launch_dtrdt_step(const StepArgs &a, bool any_random, cudaStream_t st);

// DTrDT thread cells other than 4 x 4 sites (cells.cu): whether a cell shape
// has a kernel, and the launch of one device step with it.
bool cells_shape_supported(int cx, int cy);
cudaError_t launch_cells_step(const StepArgs &a, bool any_random, cudaStream_t st);

// Adds one to the device MCS counter.
cudaError_t launch_advance_t(uint32_t *t_ptr, cudaStream_t st);

// Flat start h = (x+y) mod 2 on the planar lattice (or on `rows` rows from an
// even lattice row on, bit planes of `rows` rows each).
cudaError_t launch_init_flat(uint32_t *lat, uint32_t L, cudaStream_t st);
cudaError_t launch_init_flat_rows(uint32_t *lat, uint32_t L, uint32_t rows, cudaStream_t st);

// Exact roughness sums.
struct W2RowSums {
    long long r1;  // sum over x of r(x), r(x) = h(x,y) - h(0,y)
    long long r2;  // sum over x of r(x)^2
    int rmin, rmax;
    int c;         // Y(0, y)
    int pad;
};
struct W2Result {
    long long s1;
    unsigned long long s2_lo, s2_hi;
    long long hmax;
    long long lo, hi;  // extremes of the heights (relative to the first row's h(0, .))
    long long e_last;  // h(0, .) of the last row
    long long f0;      // 2 Y(0, first row) - 1
};
cudaError_t launch_w2(const uint32_t *lat, uint32_t L, W2RowSums *rows, W2Result *out,
                      cudaStream_t st);
// The same over the first nrows rows of a buffer whose bit planes hold
// plane_rows rows each (a strip of a lattice split over devices).
cudaError_t launch_w2_rows(const uint32_t *lat, uint32_t L, uint32_t nrows, uint32_t plane_rows, W2RowSums *rows,
                           W2Result *out, cudaStream_t st);

// Two-time autocorrelation sums of lattice lat_t against lat_s (both planar, L x L).
struct AcRowSums {
    long long rt, rs;  // sum over x of r_t(x), r_s(x), r(x) = h(x,y) - h(0,y)
    long long rts;     // sum over x of r_t(x) r_s(x)
    int ct, cs;        // Y(0, y) of each lattice
    int nx, ny;        // popcounts of X_t & X_s and Y_t & Y_s in row y
    int mt, ms;        // popcounts of X and Y in row y of each lattice
};
struct AcResult {
    long long sum_ht, sum_hs;                // sum h(t), sum h(s)
    unsigned long long cross_lo, cross_hi;   // sum h(t) h(s), two's-complement 128-bit
    long long occ_x, occ_y, m_t, m_s;
};
cudaError_t launch_two_time(const uint32_t *lat_t, const uint32_t *lat_s, uint32_t L, AcRowSums *rows,
                            AcResult *out, cudaStream_t st);
// C_h and C_s of an oct_ac from the exact sums of an L x L pair (numerators in
// 128-bit integers); leaves out->t and out->s to the caller.
void fill_ac(int64_t L, const AcResult &r, oct_ac *out);

// Canonical 4x4-per-word layout conversion for canonical word rows
// [cy0, cy0 + ncy) (each canonical row covers 4 lattice rows).
cudaError_t launch_pack_canonical(const uint32_t *lat, uint32_t L, uint32_t cy0, uint32_t ncy,
                                  uint32_t *out, cudaStream_t st);
cudaError_t launch_unpack_canonical(const uint32_t *in, uint32_t L, uint32_t cy0, uint32_t ncy,
                                    uint32_t *lat, cudaStream_t st);

// Sums of the kNetSlots flip counters into out[0], of the draw counters into
// out[1] and of the tail-block counters into out[2].
cudaError_t launch_net_sum(const unsigned long long *net, const unsigned long long *draws,
                           const unsigned long long *tails, long long *out, cudaStream_t st);

// Integer-pipe probe (op 0: LOP3, op 1: IMAD): operations per SM per clock
// and the SM clock during the probe.
cudaError_t measure_int_rate(int op, int sms, double *ops_per_clk_per_sm, double *mhz);

// Records the message oct_last_error() returns on this thread.
void set_last_error(const std::string &msg);

}  // namespace oct
