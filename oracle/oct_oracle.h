/*
 * CPU oracle for the octahedron-model DTrDT simulation (test infrastructure).
 *
 * This header and oct_oracle.c are the plain, slow, obviously-correct
 * statement of what the GPU path computes.  Only the test-suite, the smoke
 * check and the benchmark's CPU-baseline leg may load this library.  It
 * shares no code, header, table or constant generator with the CUDA path.
 *
 * Lattice representation used by every oracle routine: two byte arrays X and
 * Y of L*L entries, index y*L + x, each entry 0 or 1:
 *   X[y*L+x] = 1  iff  h(x,y) - h(x-1,y) = +1   (slope to the left neighbour)
 *   Y[y*L+x] = 1  iff  h(x,y) - h(x,y-1) = +1   (slope to the lower neighbour)
 * with periodic indices.  This is the paper's on-site slope convention
 * (Sec. 3, dead-border scheme: each site carries the slope towards its left
 * neighbour; updates only reach the +x and +y neighbours).
 *
 * Parity status of each routine is listed in oct_oracle.c next to the code.
 */
#ifndef OCT_ORACLE_H
#define OCT_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Stream tags (top 4 bits of counter word 3). */
#define OO_TAG_MCS 1u
#define OO_TAG_SET 2u
#define OO_TAG_SITE 3u
#define OO_TAG_ACC 4u
#define OO_TAG_SEQ 5u
#define OO_TAG_REPLICA 6u
#define OO_TAG_TAIL 7u
#define OO_TAG_SITE_DB 8u
#define OO_TAG_BORG 9u  /* block-layer origin of DTrDTr */

/* Block-layer schemes (Sec. 3.1). */
#define OO_SCHEME_DT 0          /* single-hit double tiling (DTrDT)                     */
#define OO_SCHEME_DB 1          /* single-hit dead border, delayed borders (DTrDB)      */
#define OO_SCHEME_DB_IGNORE 2   /* dead border with border attempts not delayed         */
#define OO_SCHEME_DTR 3         /* double tiling with a random block-layer origin (DTrDTr) */

typedef struct {
    int64_t L;        /* lateral size; periodic */
    int64_t Bx, By;   /* device-layer sub-tile size in sites (device tile = 2Bx x 2By) */
    int64_t cx, cy;   /* block-layer thread-cell size in sites */
    double p, q;      /* deposition / removal probabilities, Eq. (1) */
    uint64_t seed;    /* Philox key = (seed low 32 bits, seed high 32 bits) */
    int64_t scheme;   /* OO_SCHEME_*; 0 = DTrDT */
} oo_params;

/* Philox-4x32-10 (Salmon et al., SC'11), counter ctr[4], key key[2]. */
void oo_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);

/* Acceptance threshold: accept iff u < P32, u a uniform 32-bit word. */
uint64_t oo_threshold32(double p);

/* Flat initial condition h(x,y) = (x+y) mod 2. */
void oo_init_flat(int64_t L, uint8_t *X, uint8_t *Y);

/* One Kawasaki attempt at site (x,y), Eq. (1).  Returns +1 for an accepted
 * deposition, -1 for an accepted removal, 0 otherwise.  kind_out (optional)
 * receives +1 if the site was a local minimum, -1 if a maximum, 0 otherwise.
 * u is the attempt's 32-bit uniform; it is only read when the relevant
 * probability lies strictly between 0 and 1. */
int oo_attempt(int64_t L, uint8_t *X, uint8_t *Y, int64_t x, int64_t y,
               double p, double q, uint32_t u, int *kind_out);

/* Site classification only: +1 local minimum, -1 local maximum, 0 neither. */
int oo_site_kind(int64_t L, const uint8_t *X, const uint8_t *Y, int64_t x, int64_t y);

/* O1: true random-sequential updating, n_mcs sweeps of L*L attempts starting
 * at MCS index t0.  Adds accepted depositions minus removals to *net_flips. */
void oo_seq_rs(int64_t L, double p, double q, uint64_t seed, uint8_t *X, uint8_t *Y,
               uint32_t t0, uint32_t n_mcs, int64_t *net_flips);

/* O1 on many independent seeds of one small lattice (seed0 + r for run r),
 * writing every final lattice to Xout/Yout (n_runs * L*L bytes each). */
void oo_seq_rs_many(int64_t L, double p, double q, uint64_t seed0, int64_t n_runs,
                    uint32_t n_mcs, uint8_t *Xout, uint8_t *Yout);

/* Validates a DTrDT parameter set; returns 0 if usable by the oracle. */
int oo_check_params(const oo_params *prm);

/* The per-MCS device-layer draw: origin (ox,oy) and the permutation perm[4]
 * of the four sub-tile sets. */
void oo_mcs_draw(const oo_params *prm, uint32_t t, int64_t *ox, int64_t *oy, int perm[4]);

/* O2: replay of the DTrDT schedule for n_mcs sweeps starting at MCS t0.
 * Optional instrumentation (pass NULL to skip):
 *   attempts[L*L]  : incremented for every attempted site
 *   conflicts      : if non-NULL, every read/written slope bit is tracked and
 *                    *conflicts counts bits touched by two different thread
 *                    cells in one collective step, or by two sub-tiles in one
 *                    device step (must stay 0).
 * Returns 0, or -1 on invalid parameters. */
int oo_dtrdt_run(const oo_params *prm, uint8_t *X, uint8_t *Y, uint32_t t0, uint32_t n_mcs,
                 int64_t *net_flips, int64_t *attempts, int64_t *conflicts);

/* O2 on many independent seeds (seed0 + r) of one lattice from the flat
 * start, writing every final lattice to Xout/Yout (n_runs * L*L bytes each). */
int oo_dtrdt_many(const oo_params *prm, uint64_t seed0, int64_t n_runs, uint32_t n_mcs,
                  uint8_t *Xout, uint8_t *Yout);

/* The acceptance randomness O2 uses: the four leading bits (31..28) of the
 * uniform of the thread cell at position pos (= 4*j + m) of group g at
 * collective step s, device step k, tile T, MCS t; and word i of the
 * tail stream of group g in a device step (its top 28 bits complete a uniform
 * whose leading bits tie with P32's). */
uint32_t oo_dtrdt_acc_prefix(uint64_t seed, uint32_t t, uint32_t k, uint32_t T, uint32_t g,
                             uint32_t s, int pos);
uint32_t oo_dtrdt_tail_word(uint64_t seed, uint32_t t, uint32_t k, uint32_t T, uint32_t g, uint32_t i);

/* O2 restricted to a window: the lattice is only known on a W x H window whose
 * lower-left corner is the global site (wx, wy) (periodic in L).  Xw/Yw hold
 * the window, index j*W + i for global site ((wx+i) mod L, (wy+j) mod L).
 * Runs MCS t and updates every sub-tile whose footprint (sub-tile plus its +x
 * column and +y row) lies inside the window; other sub-tiles are skipped, so
 * only sites far enough from the window edge end up exact. */
int oo_dtrdt_mcs_window(const oo_params *prm, uint32_t t, int64_t wx, int64_t wy,
                        int64_t W, int64_t H, uint8_t *Xw, uint8_t *Yw, int64_t *net_flips);

/* Device step k of MCS t on one row strip of the multi-GPU partition: the
 * device-tile rows whose first row (oy + 2By ty) mod L lies in [a, a + Hs)
 * are updated.  Xs/Ys hold `rows` full rows from global row a on (index
 * j*L + x for global row (a + j) mod L), which must cover the sub-tiles of
 * those tile rows and their +y halo row.  Adds the net flips.  Returns 0, -1
 * for invalid parameters, -2 if a sub-tile reaches past the held rows. */
int oo_device_step_strip(const oo_params *P, uint32_t t, uint32_t k, int64_t a, int64_t Hs, int64_t rows,
                         uint8_t *Xs, uint8_t *Ys, int64_t *net_flips);

/* Local sites (lx[i], ly[i]) in the sub-tile of the attempts of every thread
 * cell i = (TC row)*(Bx/cx) + (TC column) in collective step s of sub-tile T,
 * device step k, MCS t (the block layer's site selection alone, for tests of
 * the attempt pattern).  Returns 0, or -1 for invalid parameters. */
int oo_subtile_step_sites(const oo_params *P, uint32_t t, uint32_t k, uint32_t T, int64_t s,
                          int64_t *lx, int64_t *ly);

/* The first n_steps collective steps of one sub-tile alone (Bx x By sites at
 * (x0, y0), periodic in L), device step k, tile index T, MCS t, once for each
 * seed seed0 + r, r < n_runs, each from the lattice (X0, Y0).  Writes each
 * resulting lattice to Xout/Yout (n_runs * L*L bytes each) and its net flips
 * to net_flips[r] (optional).  The tail stream starts from word 0, as at the
 * start of a device step.  For exact one-step distributions in the tests.
 * Returns 0, or -1 for invalid parameters. */
int oo_subtile_steps_many(const oo_params *P, uint64_t seed0, int64_t n_runs, uint32_t t, uint32_t k,
                          uint32_t T, int64_t x0, int64_t y0, int64_t n_steps, const uint8_t *X0,
                          const uint8_t *Y0, uint8_t *Xout, uint8_t *Yout, int64_t *net_flips);

/* Plants one of two known mistakes in the block layer, for negative controls
 * of the tests only: 1 = thread cells 2i and 2i+1 of a band read the same
 * site-draw bits; 2 = DTrDB carries out corner attempts before border
 * attempts; 3 = every group's tied candidates take words from group 0's tail
 * stream.  0 (the default) plants nothing.  Not thread-safe; a test sets it
 * and resets it to 0. */
void oo_set_plant(int which);

/* Records, for the tests, the tail word every tied candidate takes (the
 * candidates whose four leading uniform bits equal those of P32): four int64
 * per tie in buf (stream group, word index, candidate group, position 4j+m),
 * at most cap ties, in the order they are taken.  buf = NULL stops recording.
 * oo_tie_log_count() returns the number recorded.  Not thread-safe. */
void oo_set_tie_log(int64_t *buf, int64_t cap);
int64_t oo_tie_log_count(void);

/* O3: exact roughness sums, Eq. (3).  Heights relative to h(0,0) = 0 are
 * integrated first up column 0 and then along each row.  s1 = sum h,
 * s2 = sum h^2 returned as two 64-bit halves of an unsigned 128-bit value
 * (s2 is non-negative), hmax = max |h|. */
void oo_w2_sums(int64_t L, const uint8_t *X, const uint8_t *Y, int64_t *s1,
                uint64_t *s2_lo, uint64_t *s2_hi, int64_t *hmax);

/* Same sums, integrating first along row 0 and then up each column. */
void oo_w2_sums_colfirst(int64_t L, const uint8_t *X, const uint8_t *Y, int64_t *s1,
                         uint64_t *s2_lo, uint64_t *s2_hi);

/* W^2 = (N*S2 - S1^2)/N^2 from exact integer sums, N = L*L. */
double oo_w2_from_sums(int64_t L, int64_t s1, uint64_t s2_lo, uint64_t s2_hi);

/* Invariants of the slope lattice.  Returns a bit set of violated properties:
 *   1: some row does not hold exactly L/2 up-slopes in X
 *   2: some column does not hold exactly L/2 up-slopes in Y
 *   4: some plaquette has non-zero height circulation
 * (0 = all hold). */
int oo_invariants(int64_t L, const uint8_t *X, const uint8_t *Y);

/* Canonical exchange layout: one 32-bit word per 4x4 block of sites, word
 * index (y/4)*(L/4) + x/4, bit 2*(4*(y%4) + x%4) = X, the next bit = Y. */
void oo_pack_canonical(int64_t L, const uint8_t *X, const uint8_t *Y, uint32_t *words);
void oo_unpack_canonical(int64_t L, const uint32_t *words, uint8_t *X, uint8_t *Y);

/* O3 and the invariant checks on a bit-packed planar lattice (X plane then
 * Y plane, L rows of L/32 words, bit x%32 of word x/32 is site x).  The
 * circulation check covers rows [circ_y0, circ_y1). */
void oo_w2_sums_planar(int64_t L, const uint32_t *words, int64_t *s1, uint64_t *s2_lo,
                       uint64_t *s2_hi, int64_t *hmax);
int oo_invariants_planar(int64_t L, const uint32_t *words, int64_t circ_y0, int64_t circ_y1);

/* Two-time quantities of Sec. 2 (Eq. (5) and the slope and height forms
 * C_s, C_h that follow it) for one sample: lattice (Xt, Yt) at time t and
 * (Xs, Ys) at the waiting time s.  Heights of each lattice are relative to
 * its own h(0,0) = 0; the covariance does not depend on that choice.
 *   sum_ht = sum h(t),  sum_hs = sum h(s),  cross = sum h(t) h(s)  (128-bit)
 *   occ_x  = sum X_t X_s,  occ_y = sum Y_t Y_s   (lattice-gas occupations)
 *   m_t    = sum (X_t + Y_t),  m_s = sum (X_s + Y_s)
 * parity unpinned: no; pinned by tests/test_oracle_two_time.py. */
typedef struct {
    int64_t sum_ht, sum_hs;
    uint64_t cross_lo;
    int64_t cross_hi;
    int64_t occ_x, occ_y;
    int64_t m_t, m_s;
} oo_two_time;

void oo_two_time_sums(int64_t L, const uint8_t *Xt, const uint8_t *Yt, const uint8_t *Xs,
                      const uint8_t *Ys, oo_two_time *out);

/* C_h(t,s) = <h(t) h(s)> - <h(t)><h(s)> with <.> the mean over the N = L*L
 * sites: (N*cross - sum_ht*sum_hs) / N^2, numerator in 128-bit integers.
 * C_s(t,s) = <n(t) n(s)> - <n(t)><n(s)> over the 2N slope variables (x and y):
 * (2N*(occ_x+occ_y) - m_t*m_s) / (2N)^2. */
double oo_ch_from_sums(int64_t L, const oo_two_time *a);
double oo_cs_from_sums(int64_t L, const oo_two_time *a);

/* Per-replica key derivation for batched runs: key_r = the first two words of
 * Philox(master key, (r, 0, 0, TAG_REPLICA << 28)). */
uint64_t oo_replica_seed(uint64_t master_seed, uint32_t r);

#ifdef __cplusplus
}
#endif
#endif
