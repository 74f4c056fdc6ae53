/*
 * CPU oracle for the octahedron-model DTrDT simulation.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, the smoke check and the
 * benchmark's CPU-baseline / reference legs load this library.  The product
 * path (the CUDA library and its binding) never calls it, and the two share
 * no code: this file is compiled on its own with gcc.
 *
 * Every routine is written for clarity, one site and one attempt at a time,
 * in the order the paper states the method:
 *   - the model and its update rule: Sec. 2.1, Eq. (1);
 *   - the roughness: Eq. (3) (mean over the L^2 sites, see below);
 *   - one MCS = one sweep = L^2 attempts: Sec. 2.1, definition of the MCS;
 *   - random-sequential dynamics (O1): Sec. 1 (RS site selection);
 *   - DTrDT (O2): device layer = double tiling with a random origin
 *     (Sec. 3, "DT" and "DTr"; Fig. 2); block layer = single-hit double
 *     tiling, one randomly drawn domain set per collective step
 *     (Sec. 3.1, block layer paragraph);
 *   - the other block layers: single-hit dead border with delayed borders
 *     (DTrDB, Sec. 3.1, delayed borders; Fig. 5) and double tiling whose origin moves after
 *     every collective step (DTrDTr, Sec. 4.1.2);
 *   - two-time autocorrelations C_h, C_s: Sec. 2, Eq. (5).
 * Where the paper is silent (random-number streams, thread-cell units,
 * acceptance rounding), a reading is fixed here and restated at each use.
 *
 * Parity pins (tests/test_oracle_*.py): Philox known-answer vectors and an
 * independent Philox implementation; flat-start closed forms; lattice
 * invariants after every run; exact 4x4 master equations for O1 and for O2
 * (degenerate 2x2 thread cells); site-selection and acceptance statistics
 * for O2 at full thread-cell size; every cell's site against an independent
 * statement of the site fields, and neighbouring cells' offsets jointly
 * uniform, at 4x4 to 32x16 cells; exact one-collective-step distributions of
 * DT, DTrDB (delayed borders) and DTrDTr on sub-tiles of several cells;
 * planted-mistake tests of the checker and of the block layer (oo_set_plant).
 */
#include "oct_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

typedef unsigned __int128 u128;
typedef __int128 i128;

/* ------------------------------------------------------------------------ */
/* Philox-4x32-10, Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as  */
/* easy as 1, 2, 3", SC'11: ten rounds of two 32x32->64 multiplications     */
/* with the round constants below and a Weyl-sequence key schedule.         */
/* ------------------------------------------------------------------------ */
void oo_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        uint64_t prod0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
        uint64_t prod1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(prod0 >> 32), lo0 = (uint32_t)prod0;
        uint32_t hi1 = (uint32_t)(prod1 >> 32), lo1 = (uint32_t)prod1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0;
        c1 = n1;
        c2 = n2;
        c3 = n3;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    out[0] = c0;
    out[1] = c1;
    out[2] = c2;
    out[3] = c3;
}

static void seed_key(uint64_t seed, uint32_t key[2]) {
    key[0] = (uint32_t)(seed & 0xFFFFFFFFu);
    key[1] = (uint32_t)(seed >> 32);
}

static void philox_at(const uint32_t key[2], uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                      uint32_t out[4]) {
    uint32_t ctr[4] = {c0, c1, c2, c3};
    oo_philox4x32_10(ctr, key, out);
}

/* Acceptance: the paper gives probabilities p, q (Eq. (1)) but no rounding.
 * Reading: P32 = floor(p * 2^32) (exact: scaling a double by 2^32 is exact),
 * accept iff the attempt's uniform 32-bit word u < P32; p = 1 always accepts
 * and p = 0 never does. */
uint64_t oo_threshold32(double p) {
    if (!(p > 0.0)) return 0;
    if (p >= 1.0) return (uint64_t)1 << 32;
    return (uint64_t)floor(ldexp(p, 32));
}

static inline int64_t wrap(int64_t a, int64_t L) {
    int64_t r = a % L;
    return r < 0 ? r + L : r;
}

/* Planted mistakes, for the negative controls of the tests only (0 = none,
 * the default; see oo_set_plant in the header). */
static int g_plant = 0;

void oo_set_plant(int which) { g_plant = which; }

/* Optional record of the tail words the tied candidates take, for the tests:
 * four int64 per tie (stream group, word index, candidate group, position). */
static int64_t *g_tie_log = NULL;
static int64_t g_tie_cap = 0, g_tie_n = 0;

void oo_set_tie_log(int64_t *buf, int64_t cap) {
    g_tie_log = buf;
    g_tie_cap = buf ? cap : 0;
    g_tie_n = 0;
}

int64_t oo_tie_log_count(void) { return g_tie_n; }

/* ------------------------------------------------------------------------ */
/* Model, Sec. 2.1 / Eq. (1)                                                 */
/* ------------------------------------------------------------------------ */
void oo_init_flat(int64_t L, uint8_t *X, uint8_t *Y) {
    /* h(x,y) = (x+y) mod 2: the slope to the left/lower neighbour is +1
     * exactly where x+y is odd. */
    for (int64_t y = 0; y < L; ++y)
        for (int64_t x = 0; x < L; ++x) {
            X[y * L + x] = (uint8_t)((x + y) & 1);
            Y[y * L + x] = (uint8_t)((x + y) & 1);
        }
}

int oo_site_kind(int64_t L, const uint8_t *X, const uint8_t *Y, int64_t x, int64_t y) {
    /* Eq. (1): the 2x2 matrix lists (x-slope at s, x-slope at s+x) in the
     * first row and (y-slope at s, y-slope at s+y) in the second; [0 1;0 1]
     * is a local minimum (deposition, prob. p), [1 0;1 0] a local maximum
     * (removal, prob. q). */
    int64_t xr = wrap(x + 1, L), yu = wrap(y + 1, L);
    int xs = X[y * L + x], xn = X[y * L + xr];
    int ys = Y[y * L + x], yn = Y[yu * L + x];
    if (xs == 0 && xn == 1 && ys == 0 && yn == 1) return +1;
    if (xs == 1 && xn == 0 && ys == 1 && yn == 0) return -1;
    return 0;
}

static void flip_site(int64_t L, uint8_t *X, uint8_t *Y, int64_t x, int64_t y) {
    int64_t xr = wrap(x + 1, L), yu = wrap(y + 1, L);
    X[y * L + x] ^= 1;
    X[y * L + xr] ^= 1;
    Y[y * L + x] ^= 1;
    Y[yu * L + x] ^= 1;
}

int oo_attempt(int64_t L, uint8_t *X, uint8_t *Y, int64_t x, int64_t y, double p, double q,
               uint32_t u, int *kind_out) {
    int kind = oo_site_kind(L, X, Y, x, y);
    if (kind_out) *kind_out = kind;
    if (kind == 0) return 0;
    uint64_t thr = oo_threshold32(kind > 0 ? p : q);
    if ((uint64_t)u >= thr) return 0;
    flip_site(L, X, Y, x, y);
    return kind;
}

/* ------------------------------------------------------------------------ */
/* O1: random-sequential updating (Sec. 1): each of the L^2 attempts of an   */
/* MCS picks a site uniformly at random.  Stream: block                      */
/* Philox(seed, (a mod 2^32, a div 2^32, t, SEQ<<28)) for attempt a of MCS  */
/* t; x = (w0*L) >> 32, y = (w1*L) >> 32, u = w2.                            */
/* ------------------------------------------------------------------------ */
void oo_seq_rs(int64_t L, double p, double q, uint64_t seed, uint8_t *X, uint8_t *Y, uint32_t t0,
               uint32_t n_mcs, int64_t *net_flips) {
    uint32_t key[2];
    seed_key(seed, key);
    const int64_t N = L * L;
    int64_t net = 0;
    for (uint32_t dt = 0; dt < n_mcs; ++dt) {
        uint32_t t = t0 + dt;
        for (int64_t a = 0; a < N; ++a) {
            uint32_t w[4];
            philox_at(key, (uint32_t)a, (uint32_t)((uint64_t)a >> 32), t, OO_TAG_SEQ << 28, w);
            int64_t x = (int64_t)(((uint64_t)w[0] * (uint64_t)L) >> 32);
            int64_t y = (int64_t)(((uint64_t)w[1] * (uint64_t)L) >> 32);
            net += oo_attempt(L, X, Y, x, y, p, q, w[2], NULL);
        }
    }
    if (net_flips) *net_flips += net;
}

void oo_seq_rs_many(int64_t L, double p, double q, uint64_t seed0, int64_t n_runs, uint32_t n_mcs,
                    uint8_t *Xout, uint8_t *Yout) {
    const int64_t N = L * L;
    for (int64_t r = 0; r < n_runs; ++r) {
        uint8_t *X = Xout + r * N, *Y = Yout + r * N;
        oo_init_flat(L, X, Y);
        oo_seq_rs(L, p, q, seed0 + (uint64_t)r, X, Y, 0, n_mcs, NULL);
    }
}

/* ------------------------------------------------------------------------ */
/* O2: DTrDT                                                                 */
/* ------------------------------------------------------------------------ */
static int ilog2_exact(int64_t v) {
    int k = 0;
    if (v <= 0) return -1;
    while (((int64_t)1 << k) < v) ++k;
    return ((int64_t)1 << k) == v ? k : -1;
}

int oo_check_params(const oo_params *P) {
    if (!P) return -1;
    if (P->L < 2 || (P->L & 1)) return -1;
    if (P->L > ((int64_t)1 << 31)) return -1;
    if (ilog2_exact(P->cx) < 1 || ilog2_exact(P->cy) < 1) return -1;
    if (P->Bx < P->cx || P->By < P->cy || P->Bx % P->cx || P->By % P->cy) return -1;
    int64_t BW = P->Bx < 32 ? P->Bx : 32;
    if (P->Bx % BW || BW % P->cx || BW / P->cx > 8) return -1;
    if (P->L % (2 * P->Bx) || P->L % (2 * P->By)) return -1;
    if (!(P->p >= 0.0 && P->p <= 1.0 && P->q >= 0.0 && P->q <= 1.0)) return -1;
    if (P->cx * P->cy * 8 >= ((int64_t)1 << 30)) return -1;
    if (P->scheme < OO_SCHEME_DT || P->scheme > OO_SCHEME_DTR) return -1;
    if (P->scheme == OO_SCHEME_DTR && (P->cx > 16 || P->cy > 16)) return -1;
    int64_t groups = (P->Bx / BW) * ((P->By / P->cy + 3) / 4);
    if (groups >= ((int64_t)1 << 28)) return -1;
    int64_t tiles = (P->L / (2 * P->Bx)) * (P->L / (2 * P->By));
    if (tiles > ((int64_t)1 << 32)) return -1;
    return 0;
}

/* The index-th permutation of (0,1,2,3) in lexicographic order. */
static void perm_from_index(uint32_t index, int perm[4]) {
    int avail[4] = {0, 1, 2, 3};
    int n = 4;
    uint32_t fact[4] = {6, 2, 1, 1};
    for (int i = 0; i < 4; ++i) {
        uint32_t pick = index / fact[i];
        index %= fact[i];
        perm[i] = avail[pick];
        for (int j = (int)pick; j < n - 1; ++j) avail[j] = avail[j + 1];
        --n;
    }
}

void oo_mcs_draw(const oo_params *P, uint32_t t, int64_t *ox, int64_t *oy, int perm[4]) {
    /* Device layer (DTr): the tiling origin is moved to a uniformly random
     * site once per MCS, and the four sub-tile sets are visited in a fresh
     * uniformly shuffled order each MCS (Sec. 3, DT and DTr). */
    uint32_t key[2], M[4];
    seed_key(P->seed, key);
    philox_at(key, t, 0, 0, OO_TAG_MCS << 28, M);
    *ox = (int64_t)(((uint64_t)M[0] * (uint64_t)P->L) >> 32);
    *oy = (int64_t)(((uint64_t)M[1] * (uint64_t)P->L) >> 32);
    perm_from_index((uint32_t)(((uint64_t)M[2] * 24u) >> 32), perm);
}

/* A rectangular window of the periodic lattice. */
typedef struct {
    int64_t L, wx, wy, W, H;
    uint8_t *X, *Y;
} view_t;

static inline int64_t vidx(const view_t *v, int64_t gx, int64_t gy) {
    int64_t i = wrap(gx - v->wx, v->L), j = wrap(gy - v->wy, v->L);
    return j * v->W + i;
}

typedef struct {
    int64_t *dev_stamp, *dev_owner, *step_stamp, *step_owner; /* 2 per site: X then Y */
    int64_t *flip_stamp;                                      /* last batch that flipped the bit */
    int64_t dev_serial, step_serial, count;
} conflict_t;

static void touch(conflict_t *cf, int64_t bit, int64_t tile, int64_t tc) {
    if (!cf) return;
    if (cf->dev_stamp[bit] == cf->dev_serial && cf->dev_owner[bit] != tile) cf->count++;
    cf->dev_stamp[bit] = cf->dev_serial;
    cf->dev_owner[bit] = tile;
    if (cf->step_stamp[bit] == cf->step_serial && cf->step_owner[bit] != tc) cf->count++;
    cf->step_stamp[bit] = cf->step_serial;
    cf->step_owner[bit] = tc;
}

/* Acceptance uniforms (a reading: the paper names no generator).  The
 * uniform u of a thread cell's attempt is 32 bits, most significant first:
 *   - bits 31..28: "level" bits, positional per group: bit (31-l) of u is bit
 *     spl_off + pos of word l (l = 0..3) of Philox(seed, (t, k|((s/spl)*8)<<2,
 *     T, ACC<<28|g)), pos = 4j+m, where a group of tpb cells per 32-site band
 *     uses 4*tpb positions per step, so one block serves spl = 8/tpb = cx/4
 *     consecutive steps and step s takes positions from spl_off =
 *     (s % spl)*4*tpb on (spl = 1 for 4x4-site cells and for bands narrower
 *     than 32 sites);
 *   - bits 27..0: only needed when bits 31..28 equal those of P32 (otherwise
 *     u < P32 is already decided); they are the top 28 bits of the next word
 *     of the group's own tail stream, word i = word i%4 of
 *     Philox(seed, (t, k|(i/4)<<2, T, TAIL<<28|g)), i counted from 0 at the
 *     start of each device step; within a collective step (a DB phase) the
 *     group's candidates that need one take words in order of position pos. */
static void acc_level_words(const uint32_t key[2], uint32_t t, uint32_t k, uint32_t T, uint32_t g,
                            uint32_t s, uint32_t spl, uint32_t lw[4]) {
    philox_at(key, t, k | (((s / spl) * 8) << 2), T, (OO_TAG_ACC << 28) | g, lw);
}

/* Bits 31..28 of the uniform of the thread cell at position pos. */
static uint32_t acc_prefix(const uint32_t lw[4], int pos) {
    uint32_t hi = 0;
    for (int l = 0; l < 4; ++l) hi |= ((lw[l] >> pos) & 1u) << (3 - l);
    return hi;
}

static uint32_t tail_word(const uint32_t key[2], uint32_t t, uint32_t k, uint32_t T, uint32_t g,
                          uint32_t i) {
    uint32_t w[4];
    philox_at(key, t, k | ((i / 4) << 2), T, (OO_TAG_TAIL << 28) | g, w);
    return w[i % 4];
}

uint32_t oo_dtrdt_acc_prefix(uint64_t seed, uint32_t t, uint32_t k, uint32_t T, uint32_t g,
                             uint32_t s, int pos) {
    uint32_t key[2], w[4];
    seed_key(seed, key);
    acc_level_words(key, t, k, T, g, s, 1u, w);
    return acc_prefix(w, pos);
}

uint32_t oo_dtrdt_tail_word(uint64_t seed, uint32_t t, uint32_t k, uint32_t T, uint32_t g, uint32_t i) {
    uint32_t key[2];
    seed_key(seed, key);
    return tail_word(key, t, k, T, g, i);
}

typedef struct {
    int64_t is, ir, iu; /* view indices of s, s+x, s+y */
    int kind;           /* +1 minimum, -1 maximum */
    uint32_t g;
    int pos;
    int decided;        /* 1 accepted, 0 rejected, -1 needs a tail word */
    uint64_t thr;
    uint32_t hi;        /* leading four bits of the acceptance uniform */
    int random;         /* the probability lies strictly inside (0,1) */
    uint64_t thr_min, thr_max;
    int random_min, random_max;
    int64_t tc;         /* thread-cell index (conflict tracking) */
} attempt_t;

static int by_group_then_position(const void *pa, const void *pb) {
    const attempt_t *a = (const attempt_t *)pa, *b = (const attempt_t *)pb;
    if (a->g != b->g) return a->g < b->g ? -1 : 1;
    return (a->pos > b->pos) - (a->pos < b->pos);
}

/* Decides, flips and counts the attempts of one conflict-free batch (a
 * collective step of DT, or one phase of a DB step): attempts whose site is
 * eligible on the current state are decided by the four leading level bits of
 * their uniform; ties take the next words of their group's tail stream
 * (tail_next[g] = words group g used so far), in order of position. */
static void decide_and_flip(const uint32_t key[2], uint32_t t, uint32_t k, uint32_t T, view_t *v,
                            attempt_t *att, int64_t na, attempt_t *tied, uint32_t *tail_next,
                            int64_t *net, conflict_t *cf) {
    int64_t nt = 0;
    for (int64_t i = 0; i < na; ++i) {
        attempt_t *A = &att[i];
        A->kind = 0;
        if (v->X[A->is] == 0 && v->X[A->ir] == 1 && v->Y[A->is] == 0 && v->Y[A->iu] == 1)
            A->kind = +1;
        else if (v->X[A->is] == 1 && v->X[A->ir] == 0 && v->Y[A->is] == 1 && v->Y[A->iu] == 0)
            A->kind = -1;
        A->decided = 0;
        if (A->kind == 0) continue;
        A->thr = A->kind > 0 ? A->thr_min : A->thr_max;
        A->random = A->kind > 0 ? A->random_min : A->random_max;
        if (!A->random) {
            A->decided = A->thr > 0 ? 1 : 0; /* probability 1 or 0 */
        } else {
            const uint32_t thr_hi = (uint32_t)(A->thr >> 28);
            A->decided = A->hi < thr_hi ? 1 : (A->hi > thr_hi ? 0 : -1);
            if (A->decided < 0) tied[nt++] = *A;
        }
    }
    qsort(tied, (size_t)nt, sizeof(attempt_t), by_group_then_position);
    for (int64_t i = 0; i < nt; ++i) {
        /* the candidate's own group's stream (planted mistake 3: group 0's for all) */
        const uint32_t gs = g_plant == 3 ? 0u : tied[i].g;
        const uint32_t wi = tail_next[gs]++;
        if (g_tie_log && g_tie_n < g_tie_cap) {
            int64_t *e = g_tie_log + 4 * g_tie_n++;
            e[0] = gs;
            e[1] = wi;
            e[2] = tied[i].g;
            e[3] = tied[i].pos;
        }
        const uint32_t low28 = tail_word(key, t, k, T, gs, wi) >> 4;
        tied[i].decided = (uint64_t)low28 < (tied[i].thr & 0x0FFFFFFFu) ? 1 : 0;
    }
    /* apply the accepted flips (no two share a bit; tracked when cf is set) */
    for (int64_t i = 0; i < na + nt; ++i) {
        const attempt_t *A = i < na ? &att[i] : &tied[i - na];
        if (A->decided != 1) continue;
        if (cf) {
            const int64_t nv = v->W * v->H;
            const int64_t bits[4] = {A->is, A->ir, nv + A->is, nv + A->iu};
            for (int b = 0; b < 4; ++b) {
                if (cf->flip_stamp[bits[b]] == cf->step_serial) cf->count++;
                cf->flip_stamp[bits[b]] = cf->step_serial;
            }
        }
        v->X[A->is] ^= 1;
        v->X[A->ir] ^= 1;
        v->Y[A->is] ^= 1;
        v->Y[A->iu] ^= 1;
        *net += A->kind;
    }
}

/* Block layer on one sub-tile.
 *
 * The sub-tile (Bx x By sites, local origin (x0,y0)) is cut into thread
 * cells (TC) of cx x cy sites.  Per collective step every TC performs exactly
 * one attempt (single hit), then all synchronise; cx*cy collective steps make
 * one sweep of the sub-tile (Bx*By attempts).
 *
 * DT (double tiling): each TC is cut into four sub-cells of (cx/2) x (cy/2)
 * sites, sub-cell d = (dx,dy) = (d&1, d>>1); per step the block draws d
 * uniformly (with replacement, not a permutation) and every TC attempts a
 * uniform site of its sub-cell d.  Attempts of one step never share a slope
 * bit, so every decision is taken on the state before the step.
 *
 * DB (dead border): every TC attempts a uniform site of its whole cell.  The
 * cell's last column (x = cx-1) and last row (y = cy-1) form its border,
 * since an update there reaches the next cell.  With delayed borders, bulk
 * attempts are carried out first, then border attempts, and attempts at the
 * corner (cx-1, cy-1), which touch two borders, last; each phase is
 * conflict-free and sees the flips of the earlier ones.  The paper delays
 * borders only when both p and q are non-zero; with one of them zero two
 * neighbouring sites are never both accepted, and its DB runs carry out all
 * attempts of a step together (a reading of Sec. 3.1: DB does
 * the same).  DB_IGNORE carries out all attempts together for any p, q; with
 * both non-zero two accepted flips can then hit the same slope bit, which the
 * flip tracker counts.
 *
 * DTR (DTrDTr, Sec. 4.1.2): DT whose block-layer origin
 * moves to a uniform (ax, ay) in [0,cx) x [0,cy) after every collective step,
 * the cell grid wrapping around the sub-tile.  The active sub-cell of set d
 * then starts at column c0 = (ax + dx*cx/2) mod cx and row r0 = (ay +
 * dy*cy/2) mod cy of every (unshifted) cell; the attempt of TC (a, c) is at
 * ((a*cx + c0 + rx) mod Bx, (c*cy + r0 + ry) mod By).  (Each shifted cell is
 * labelled by the unshifted cell holding the first site of its active
 * sub-cell; a relabelling of cells does not change the dynamics.)
 *
 * Random streams (a reading: the paper names no generator):
 *   block origin (DTR) for step s : byte s%4 of word (s%16)/4 of
 *                         Philox(seed, (t, k|(s/16)<<2, T, BORG<<28)); ax =
 *                         its low log2(cx) bits, ay = log2(cy) bits from bit 4.
 *   set draw (DT) for step s : word (s%64)/16 of Philox(seed, (t, k|(s/64)<<2, T, SET<<28)),
 *                         bits 2*(s%16) .. +1.
 *   TCs are grouped: a band is one TC row, BW = min(32,Bx) sites wide; a group
 *   is four vertically consecutive bands of one band column; g = (c/4)*(Bx/BW)
 *   + band column, m = c%4 (c = TC row), j = TC index inside its band.
 *   site draw           : word m of Philox(seed, (t, k|(s/spw)<<2, T, TAG<<28|g)),
 *                         TAG = SITE (DT) or SITE_DB (DB), bits fw*j +
 *                         (s%spw)*(fw/spw) .. + bpt-1 (bpt = log2 of the
 *                         sub-cell (DT) or cell (DB) area), low bits = x offset.
 *   acceptance uniform  : see acc_level_words / tail_word above; with DB the
 *                         tail words are taken phase by phase.
 */
/* The block-layer draws of one collective step that every TC of the
 * sub-tile shares: the DT set (dx, dy) and, for DTR, the block origin. */
typedef struct {
    int64_t dx, dy;  /* sub-cell set d = (dx, dy) (DT, DTR) */
    int64_t c0, r0;  /* first column / row of the active sub-cell in each cell */
} step_draw_t;

static step_draw_t step_draw(const oo_params *P, const uint32_t key[2], uint32_t t, uint32_t k,
                             uint32_t T, int64_t s) {
    step_draw_t d = {0, 0, 0, 0};
    if (P->scheme == OO_SCHEME_DB || P->scheme == OO_SCHEME_DB_IGNORE) return d;
    uint32_t sw[4];
    philox_at(key, t, k | (uint32_t)((s / 64) << 2), T, OO_TAG_SET << 28, sw);
    const int set = (int)((sw[(s % 64) / 16] >> (2 * (s % 16))) & 3u);
    d.dx = set & 1;
    d.dy = set >> 1;
    d.c0 = d.dx * (P->cx / 2);
    d.r0 = d.dy * (P->cy / 2);
    if (P->scheme == OO_SCHEME_DTR) {
        uint32_t bw[4];
        philox_at(key, t, k | (uint32_t)((s / 16) << 2), T, OO_TAG_BORG << 28, bw);
        const uint32_t byte = (bw[(s % 16) / 4] >> (8 * (s % 4))) & 0xFFu;
        const int64_t ax = byte & (uint32_t)(P->cx - 1), ay = (byte >> 4) & (uint32_t)(P->cy - 1);
        d.c0 = (ax + d.c0) % P->cx;
        d.r0 = (ay + d.r0) % P->cy;
    }
    return d;
}

/* The field of the site word that TC j of a band reads: its own (planted
 * mistake 1 makes cells 2i and 2i+1 share the field of cell 2i). */
static int64_t site_field(int64_t j) { return g_plant == 1 ? (j & ~(int64_t)1) : j; }

/* Local site in the sub-tile of the attempt of TC column a, TC row c, whose
 * random offset inside its sub-cell (DT, DTR) or cell (DB) is (rx, ry). */
static void tc_local_site(const oo_params *P, const step_draw_t *d, int64_t a, int64_t c, int64_t rx,
                          int64_t ry, int64_t *lx, int64_t *ly) {
    *lx = (a * P->cx + d->c0 + rx) % P->Bx;
    *ly = (c * P->cy + d->r0 + ry) % P->By;
}

static void run_subtile(const oo_params *P, const uint32_t key[2], uint32_t t, uint32_t k,
                        uint32_t T, int64_t x0, int64_t y0, view_t *v, int64_t *net,
                        int64_t *attempts, conflict_t *cf, int64_t s_end) {
    const int64_t L = P->L, Bx = P->Bx, By = P->By, cx = P->cx, cy = P->cy;
    const int db = P->scheme == OO_SCHEME_DB || P->scheme == OO_SCHEME_DB_IGNORE;
    /* The paper delays border attempts only where two neighbouring sites can
     * both be accepted, i.e. when both p and q are non-zero; with one of them
     * zero its DB runs carry out all attempts of a step together. */
    const int delayed = P->scheme == OO_SCHEME_DB && P->p > 0.0 && P->q > 0.0;
    const int64_t BW = Bx < 32 ? Bx : 32;
    const int64_t tcs_per_band = BW / cx;
    const int64_t band_cols = Bx / BW;
    const int64_t tc_rows = By / cy;
    const int64_t group_rows = (tc_rows + 3) / 4;
    const int64_t ux = db ? cx : cx / 2, uy = db ? cy : cy / 2; /* the region a TC draws from */
    const int bx_bits = ilog2_exact(ux), by_bits = ilog2_exact(uy);
    const int bpt = bx_bits + by_bits;
    const int64_t fw = 32 / tcs_per_band;
    const int spw = (bpt > 0 && 2 * bpt <= fw) ? 2 : 1;
    /* steps served by one level block: cx/4 in 32-site bands, else 1 */
    const uint32_t spl_acc = BW == 32 ? (uint32_t)(8 / tcs_per_band) : 1u;
    const uint32_t site_tag = db ? OO_TAG_SITE_DB : OO_TAG_SITE;
    const int64_t n_steps = cx * cy;
    const uint64_t thr_p = oo_threshold32(P->p), thr_q = oo_threshold32(P->q);
    const int p_random = P->p > 0.0 && P->p < 1.0;
    const int q_random = P->q > 0.0 && P->q < 1.0;
    const int64_t n_tc = (Bx / cx) * (By / cy);
    attempt_t *all = (attempt_t *)malloc(sizeof(attempt_t) * (size_t)n_tc);
    attempt_t *phase = (attempt_t *)malloc(sizeof(attempt_t) * (size_t)n_tc);
    attempt_t *tied = (attempt_t *)malloc(sizeof(attempt_t) * (size_t)n_tc);
    int *cls = (int *)malloc(sizeof(int) * (size_t)n_tc);
    /* tail-stream words each group used so far in this device step */
    uint32_t *tail_next = (uint32_t *)calloc((size_t)(group_rows * band_cols), sizeof(uint32_t));

    if (s_end > n_steps) s_end = n_steps;
    for (int64_t s = 0; s < s_end; ++s) {
        const step_draw_t sd = step_draw(P, key, t, k, T, s);
        int64_t na = 0;
        /* every thread cell's attempt: site and leading acceptance bits */
        for (int64_t gr = 0; gr < group_rows; ++gr) {
            for (int64_t bc = 0; bc < band_cols; ++bc) {
                const uint32_t g = (uint32_t)(gr * band_cols + bc);
                uint32_t site_w[4] = {0, 0, 0, 0};
                if (bpt > 0)
                    philox_at(key, t, k | (uint32_t)((s / spw) << 2), T, (site_tag << 28) | g, site_w);
                uint32_t lw[4];
                acc_level_words(key, t, k, T, g, (uint32_t)s, spl_acc, lw);
                for (int64_t m = 0; m < 4; ++m) {
                    const int64_t c = 4 * gr + m; /* TC row */
                    if (c >= tc_rows) break;
                    for (int64_t j = 0; j < tcs_per_band; ++j) {
                        const int64_t a = bc * tcs_per_band + j; /* TC column */
                        int64_t rx = 0, ry = 0;
                        if (bpt > 0) {
                            const int64_t off = fw * site_field(j) + (s % spw) * (fw / spw);
                            const uint32_t r = (site_w[m] >> off) & ((1u << bpt) - 1u);
                            rx = r & ((1u << bx_bits) - 1u);
                            ry = r >> bx_bits;
                        }
                        int64_t lx, ly;
                        tc_local_site(P, &sd, a, c, rx, ry, &lx, &ly);
                        const int64_t gx = wrap(x0 + lx, L), gy = wrap(y0 + ly, L);
                        if (attempts) attempts[gy * L + gx]++;
                        attempt_t *A = &all[na];
                        A->is = vidx(v, gx, gy);
                        A->ir = vidx(v, gx + 1, gy);
                        A->iu = vidx(v, gx, gy + 1);
                        A->g = g;
                        A->pos = (int)(4 * j + m);
                        A->hi = acc_prefix(lw, (int)((s % spl_acc) * 4 * tcs_per_band) + A->pos);
                        A->thr_min = thr_p;
                        A->thr_max = thr_q;
                        A->random_min = p_random;
                        A->random_max = q_random;
                        A->tc = c * (Bx / cx) + a;
                        /* DB phase: 0 bulk, 1 border, 2 corner (DT, ignored borders: all 0) */
                        const int on_x = (rx == cx - 1), on_y = (ry == cy - 1);
                        cls[na] = delayed ? on_x + on_y : 0;
                        ++na;
                    }
                }
            }
        }
        /* bulk, border, corner (planted mistake 2: corner before border) */
        const int order[3] = {0, g_plant == 2 ? 2 : 1, g_plant == 2 ? 1 : 2};
        for (int pi = 0; pi < 3; ++pi) {
            const int ph = order[pi];
            int64_t np = 0;
            for (int64_t i = 0; i < na; ++i)
                if (cls[i] == ph) phase[np++] = all[i];
            if (np == 0) continue;
            if (cf) {
                cf->step_serial++;
                /* DT and delayed DB phases: no bit is even read by two thread
                 * cells; DB with borders carried out together: only flips are
                 * disjoint (checked in decide_and_flip) */
                const int64_t nv = v->W * v->H;
                if (!db || delayed)
                    for (int64_t i = 0; i < np; ++i) {
                        touch(cf, phase[i].is, T, phase[i].tc);
                        touch(cf, phase[i].ir, T, phase[i].tc);
                        touch(cf, nv + phase[i].is, T, phase[i].tc);
                        touch(cf, nv + phase[i].iu, T, phase[i].tc);
                    }
            }
            decide_and_flip(key, t, k, T, v, phase, np, tied, tail_next, net, cf);
        }
    }
    free(all);
    free(phase);
    free(tied);
    free(cls);
    free(tail_next);
}

int oo_subtile_step_sites(const oo_params *P, uint32_t t, uint32_t k, uint32_t T, int64_t s,
                          int64_t *lx, int64_t *ly) {
    if (oo_check_params(P) || s < 0 || s >= P->cx * P->cy) return -1;
    uint32_t key[2];
    seed_key(P->seed, key);
    const int64_t Bx = P->Bx, By = P->By, cx = P->cx, cy = P->cy;
    const int db = P->scheme == OO_SCHEME_DB || P->scheme == OO_SCHEME_DB_IGNORE;
    const int64_t BW = Bx < 32 ? Bx : 32;
    const int64_t tcs_per_band = BW / cx, band_cols = Bx / BW, tc_rows = By / cy;
    const int64_t ux = db ? cx : cx / 2, uy = db ? cy : cy / 2;
    const int bx_bits = ilog2_exact(ux), by_bits = ilog2_exact(uy);
    const int bpt = bx_bits + by_bits;
    const int64_t fw = 32 / tcs_per_band;
    const int spw = (bpt > 0 && 2 * bpt <= fw) ? 2 : 1;
    const uint32_t site_tag = db ? OO_TAG_SITE_DB : OO_TAG_SITE;
    const step_draw_t sd = step_draw(P, key, t, k, T, s);
    for (int64_t c = 0; c < tc_rows; ++c) {
        const int64_t gr = c / 4, m = c % 4;
        for (int64_t a = 0; a < Bx / cx; ++a) {
            const int64_t bc = a / tcs_per_band, j = a % tcs_per_band;
            const uint32_t g = (uint32_t)(gr * band_cols + bc);
            int64_t rx = 0, ry = 0;
            if (bpt > 0) {
                uint32_t site_w[4];
                philox_at(key, t, k | (uint32_t)((s / spw) << 2), T, (site_tag << 28) | g, site_w);
                const int64_t off = fw * site_field(j) + (s % spw) * (fw / spw);
                const uint32_t r = (site_w[m] >> off) & ((1u << bpt) - 1u);
                rx = r & ((1u << bx_bits) - 1u);
                ry = r >> bx_bits;
            }
            const int64_t i = c * (Bx / cx) + a;
            tc_local_site(P, &sd, a, c, rx, ry, &lx[i], &ly[i]);
        }
    }
    return 0;
}

int oo_subtile_steps_many(const oo_params *P, uint64_t seed0, int64_t n_runs, uint32_t t, uint32_t k,
                          uint32_t T, int64_t x0, int64_t y0, int64_t n_steps, const uint8_t *X0,
                          const uint8_t *Y0, uint8_t *Xout, uint8_t *Yout, int64_t *net_flips) {
    if (oo_check_params(P) || n_steps < 0 || n_runs < 0) return -1;
    const int64_t L = P->L, N = L * L;
    for (int64_t r = 0; r < n_runs; ++r) {
        uint8_t *X = Xout + r * N, *Y = Yout + r * N;
        memcpy(X, X0, (size_t)N);
        memcpy(Y, Y0, (size_t)N);
        uint32_t key[2];
        seed_key(seed0 + (uint64_t)r, key);
        view_t v = {L, 0, 0, L, L, X, Y};
        int64_t net = 0;
        run_subtile(P, key, t, k, T, wrap(x0, L), wrap(y0, L), &v, &net, NULL, NULL, n_steps);
        if (net_flips) net_flips[r] = net;
    }
    return 0;
}

static int footprint_inside(const view_t *v, int64_t x0, int64_t y0, int64_t Bx, int64_t By) {
    int okx = (v->W == v->L) || (wrap(x0 - v->wx, v->L) + Bx < v->W);
    int oky = (v->H == v->L) || (wrap(y0 - v->wy, v->L) + By < v->H);
    return okx && oky;
}

static void run_mcs(const oo_params *P, uint32_t t, view_t *v, int64_t *net, int64_t *attempts,
                    conflict_t *cf) {
    uint32_t key[2];
    seed_key(P->seed, key);
    int64_t ox, oy;
    int perm[4];
    oo_mcs_draw(P, t, &ox, &oy, perm);
    const int64_t tiles_x = P->L / (2 * P->Bx), tiles_y = P->L / (2 * P->By);
    for (uint32_t k = 0; k < 4; ++k) {
        /* Device step k updates the set perm[k]: quadrant (sx,sy) of every
         * 2Bx x 2By device tile.  Sub-tiles of one set never share a slope
         * bit, so their order is irrelevant (checked by the conflict
         * tracker). */
        const int sigma = perm[k];
        const int64_t sx = sigma & 1, sy = sigma >> 1;
        if (cf) cf->dev_serial++;
        for (int64_t ty = 0; ty < tiles_y; ++ty)
            for (int64_t tx = 0; tx < tiles_x; ++tx) {
                const uint32_t T = (uint32_t)(ty * tiles_x + tx);
                const int64_t x0 = wrap(ox + 2 * P->Bx * tx + P->Bx * sx, P->L);
                const int64_t y0 = wrap(oy + 2 * P->By * ty + P->By * sy, P->L);
                if (!footprint_inside(v, x0, y0, P->Bx, P->By)) continue;
                run_subtile(P, key, t, k, T, x0, y0, v, net, attempts, cf, P->cx * P->cy);
            }
    }
}

int oo_dtrdt_run(const oo_params *P, uint8_t *X, uint8_t *Y, uint32_t t0, uint32_t n_mcs,
                 int64_t *net_flips, int64_t *attempts, int64_t *conflicts) {
    if (oo_check_params(P)) return -1;
    view_t v = {P->L, 0, 0, P->L, P->L, X, Y};
    conflict_t cfs, *cf = NULL;
    const int64_t nbits = 2 * P->L * P->L;
    if (conflicts) {
        cfs.dev_stamp = (int64_t *)malloc(sizeof(int64_t) * nbits);
        cfs.dev_owner = (int64_t *)malloc(sizeof(int64_t) * nbits);
        cfs.step_stamp = (int64_t *)malloc(sizeof(int64_t) * nbits);
        cfs.step_owner = (int64_t *)malloc(sizeof(int64_t) * nbits);
        cfs.flip_stamp = (int64_t *)malloc(sizeof(int64_t) * nbits);
        if (!cfs.dev_stamp || !cfs.dev_owner || !cfs.step_stamp || !cfs.step_owner || !cfs.flip_stamp) {
            free(cfs.dev_stamp);
            free(cfs.dev_owner);
            free(cfs.step_stamp);
            free(cfs.step_owner);
            free(cfs.flip_stamp);
            return -1;
        }
        for (int64_t i = 0; i < nbits; ++i) cfs.dev_stamp[i] = cfs.step_stamp[i] = cfs.flip_stamp[i] = -1;
        cfs.dev_serial = cfs.step_serial = cfs.count = 0;
        cf = &cfs;
    }
    int64_t net = 0;
    for (uint32_t dt = 0; dt < n_mcs; ++dt) run_mcs(P, t0 + dt, &v, &net, attempts, cf);
    if (net_flips) *net_flips += net;
    if (cf) {
        *conflicts = cf->count;
        free(cfs.dev_stamp);
        free(cfs.dev_owner);
        free(cfs.step_stamp);
        free(cfs.step_owner);
        free(cfs.flip_stamp);
    }
    return 0;
}

int oo_device_step_strip(const oo_params *P, uint32_t t, uint32_t k, int64_t a, int64_t Hs, int64_t rows,
                         uint8_t *Xs, uint8_t *Ys, int64_t *net_flips) {
    /* Device step k of MCS t restricted to the device-tile rows whose first row
     * (oy + 2By ty) mod L lies in [a, a + Hs): the strip partition of the
     * multi-GPU layout.  (Xs, Ys) hold `rows` full rows from global row a on
     * (the strip and the rows below it that its sub-tiles reach). */
    if (oo_check_params(P)) return -1;
    if (Hs < 1 || rows < 1 || rows > P->L) return -1;
    uint32_t key[2];
    seed_key(P->seed, key);
    int64_t ox, oy;
    int perm[4];
    oo_mcs_draw(P, t, &ox, &oy, perm);
    const int64_t tiles_x = P->L / (2 * P->Bx), tiles_y = P->L / (2 * P->By);
    const int sigma = perm[k];
    const int64_t sx = sigma & 1, sy = sigma >> 1;
    view_t v = {P->L, 0, wrap(a, P->L), P->L, rows, Xs, Ys};
    int64_t net = 0;
    for (int64_t ty = 0; ty < tiles_y; ++ty) {
        const int64_t yt = wrap(oy + 2 * P->By * ty, P->L);
        if (wrap(yt - a, P->L) >= Hs) continue;  /* another strip's tile row */
        for (int64_t tx = 0; tx < tiles_x; ++tx) {
            const uint32_t T = (uint32_t)(ty * tiles_x + tx);
            const int64_t x0 = wrap(ox + 2 * P->Bx * tx + P->Bx * sx, P->L);
            const int64_t y0 = wrap(yt + P->By * sy, P->L);
            if (!footprint_inside(&v, x0, y0, P->Bx, P->By)) return -2;  /* strip too short */
            run_subtile(P, key, t, k, T, x0, y0, &v, &net, NULL, NULL, P->cx * P->cy);
        }
    }
    if (net_flips) *net_flips += net;
    return 0;
}

int oo_dtrdt_mcs_window(const oo_params *P, uint32_t t, int64_t wx, int64_t wy, int64_t W,
                        int64_t H, uint8_t *Xw, uint8_t *Yw, int64_t *net_flips) {
    if (oo_check_params(P)) return -1;
    if (W < 1 || H < 1 || W > P->L || H > P->L) return -1;
    view_t v = {P->L, wrap(wx, P->L), wrap(wy, P->L), W, H, Xw, Yw};
    int64_t net = 0;
    run_mcs(P, t, &v, &net, NULL, NULL);
    if (net_flips) *net_flips += net;
    return 0;
}

/* ------------------------------------------------------------------------ */
/* O3: roughness, Eq. (3).  The printed equation divides the squared mean by */
/* L rather than L^2; read as the mean over all L^2 sites (the only          */
/* translation-invariant reading).  W^2 = (N*S2 - S1^2) / N^2, N = L^2.      */
/* ------------------------------------------------------------------------ */
void oo_w2_sums(int64_t L, const uint8_t *X, const uint8_t *Y, int64_t *s1, uint64_t *s2_lo,
                uint64_t *s2_hi, int64_t *hmax) {
    i128 S1 = 0;
    u128 S2 = 0;
    int64_t hm = 0;
    int64_t h0 = 0; /* h(0,y) */
    for (int64_t y = 0; y < L; ++y) {
        if (y > 0) h0 += 2 * (int64_t)Y[y * L + 0] - 1;
        int64_t h = h0;
        for (int64_t x = 0; x < L; ++x) {
            if (x > 0) h += 2 * (int64_t)X[y * L + x] - 1;
            S1 += h;
            S2 += (u128)((i128)h * h);
            int64_t ah = h < 0 ? -h : h;
            if (ah > hm) hm = ah;
        }
    }
    *s1 = (int64_t)S1;
    *s2_lo = (uint64_t)S2;
    *s2_hi = (uint64_t)(S2 >> 64);
    if (hmax) *hmax = hm;
}

void oo_w2_sums_colfirst(int64_t L, const uint8_t *X, const uint8_t *Y, int64_t *s1,
                         uint64_t *s2_lo, uint64_t *s2_hi) {
    i128 S1 = 0;
    u128 S2 = 0;
    int64_t hx0 = 0; /* h(x,0) */
    for (int64_t x = 0; x < L; ++x) {
        if (x > 0) hx0 += 2 * (int64_t)X[0 * L + x] - 1;
        int64_t h = hx0;
        for (int64_t y = 0; y < L; ++y) {
            if (y > 0) h += 2 * (int64_t)Y[y * L + x] - 1;
            S1 += h;
            S2 += (u128)((i128)h * h);
        }
    }
    *s1 = (int64_t)S1;
    *s2_lo = (uint64_t)S2;
    *s2_hi = (uint64_t)(S2 >> 64);
}

double oo_w2_from_sums(int64_t L, int64_t s1, uint64_t s2_lo, uint64_t s2_hi) {
    const i128 N = (i128)L * L;
    const i128 S2 = (i128)(((u128)s2_hi << 64) | s2_lo);
    const i128 num = N * S2 - (i128)s1 * s1;
    return (double)num / ((double)N * (double)N);
}

/* ------------------------------------------------------------------------ */
/* Two-time autocorrelations (Sec. 2, Eq. (5) and the C_s, C_h forms after   */
/* it).  Written out site by site: both height fields are integrated exactly */
/* as in oo_w2_sums (up column 0, then along each row), and every product is */
/* accumulated in 128 bits.                                                  */
/* ------------------------------------------------------------------------ */
void oo_two_time_sums(int64_t L, const uint8_t *Xt, const uint8_t *Yt, const uint8_t *Xs,
                      const uint8_t *Ys, oo_two_time *out) {
    i128 St = 0, Ss = 0, C = 0;
    int64_t ox = 0, oy = 0, mt = 0, ms = 0;
    int64_t h0t = 0, h0s = 0; /* h(0,y) of each lattice */
    for (int64_t y = 0; y < L; ++y) {
        if (y > 0) {
            h0t += 2 * (int64_t)Yt[y * L + 0] - 1;
            h0s += 2 * (int64_t)Ys[y * L + 0] - 1;
        }
        int64_t ht = h0t, hs = h0s;
        for (int64_t x = 0; x < L; ++x) {
            const int64_t i = y * L + x;
            if (x > 0) {
                ht += 2 * (int64_t)Xt[i] - 1;
                hs += 2 * (int64_t)Xs[i] - 1;
            }
            St += ht;
            Ss += hs;
            C += (i128)ht * hs;
            ox += Xt[i] & Xs[i];
            oy += Yt[i] & Ys[i];
            mt += Xt[i] + Yt[i];
            ms += Xs[i] + Ys[i];
        }
    }
    out->sum_ht = (int64_t)St;
    out->sum_hs = (int64_t)Ss;
    out->cross_lo = (uint64_t)(u128)C;
    out->cross_hi = (int64_t)(C >> 64);
    out->occ_x = ox;
    out->occ_y = oy;
    out->m_t = mt;
    out->m_s = ms;
}

double oo_ch_from_sums(int64_t L, const oo_two_time *a) {
    const i128 N = (i128)L * L;
    const i128 cross = (i128)(((u128)(uint64_t)a->cross_hi << 64) | a->cross_lo);
    const i128 num = N * cross - (i128)a->sum_ht * a->sum_hs;
    return (double)num / ((double)N * (double)N);
}

double oo_cs_from_sums(int64_t L, const oo_two_time *a) {
    const i128 M = 2 * (i128)L * L; /* number of slope variables */
    const i128 num = M * (i128)(a->occ_x + a->occ_y) - (i128)a->m_t * a->m_s;
    return (double)num / ((double)M * (double)M);
}

/* ------------------------------------------------------------------------ */
/* Invariants fixed by the model: heights exist on the torus (row / column   */
/* slope balance, zero circulation around every plaquette).                  */
/* ------------------------------------------------------------------------ */
int oo_invariants(int64_t L, const uint8_t *X, const uint8_t *Y) {
    int bad = 0;
    for (int64_t y = 0; y < L; ++y) {
        int64_t n = 0;
        for (int64_t x = 0; x < L; ++x) n += X[y * L + x];
        if (2 * n != L) bad |= 1;
    }
    for (int64_t x = 0; x < L; ++x) {
        int64_t n = 0;
        for (int64_t y = 0; y < L; ++y) n += Y[y * L + x];
        if (2 * n != L) bad |= 2;
    }
    for (int64_t y = 0; y < L; ++y)
        for (int64_t x = 0; x < L; ++x) {
            const int64_t x1 = wrap(x + 1, L), y1 = wrap(y + 1, L);
            /* h(x+1,y)-h(x,y) + h(x+1,y+1)-h(x+1,y) - [h(x+1,y+1)-h(x,y+1)] - [h(x,y+1)-h(x,y)] */
            const int64_t circ = (2 * X[y * L + x1] - 1) + (2 * Y[y1 * L + x1] - 1) -
                                 (2 * X[y1 * L + x1] - 1) - (2 * Y[y1 * L + x] - 1);
            if (circ != 0) bad |= 4;
        }
    return bad;
}

/* ------------------------------------------------------------------------ */
/* Canonical exchange layout (paper: one 32-bit word holds 4x4 sites, two    */
/* slope bits per site; the bit order inside the word is this project's).   */
/* ------------------------------------------------------------------------ */
void oo_pack_canonical(int64_t L, const uint8_t *X, const uint8_t *Y, uint32_t *words) {
    const int64_t nw = (L / 4) * (L / 4);
    for (int64_t i = 0; i < nw; ++i) words[i] = 0;
    for (int64_t y = 0; y < L; ++y)
        for (int64_t x = 0; x < L; ++x) {
            const int64_t w = (y / 4) * (L / 4) + x / 4;
            const int b = 2 * (int)(4 * (y % 4) + (x % 4));
            words[w] |= (uint32_t)X[y * L + x] << b;
            words[w] |= (uint32_t)Y[y * L + x] << (b + 1);
        }
}

void oo_unpack_canonical(int64_t L, const uint32_t *words, uint8_t *X, uint8_t *Y) {
    for (int64_t y = 0; y < L; ++y)
        for (int64_t x = 0; x < L; ++x) {
            const int64_t w = (y / 4) * (L / 4) + x / 4;
            const int b = 2 * (int)(4 * (y % 4) + (x % 4));
            X[y * L + x] = (uint8_t)((words[w] >> b) & 1u);
            Y[y * L + x] = (uint8_t)((words[w] >> (b + 1)) & 1u);
        }
}

uint64_t oo_replica_seed(uint64_t master_seed, uint32_t r) {
    uint32_t key[2], w[4];
    seed_key(master_seed, key);
    philox_at(key, r, 0, 0, OO_TAG_REPLICA << 28, w);
    return (uint64_t)w[0] | ((uint64_t)w[1] << 32);
}

int oo_dtrdt_many(const oo_params *P, uint64_t seed0, int64_t n_runs, uint32_t n_mcs,
                  uint8_t *Xout, uint8_t *Yout) {
    if (oo_check_params(P)) return -1;
    const int64_t N = P->L * P->L;
    for (int64_t r = 0; r < n_runs; ++r) {
        oo_params Q = *P;
        Q.seed = seed0 + (uint64_t)r;
        uint8_t *X = Xout + r * N, *Y = Yout + r * N;
        oo_init_flat(P->L, X, Y);
        oo_dtrdt_run(&Q, X, Y, 0, n_mcs, NULL, NULL, NULL);
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* The same roughness sums and invariants read straight from a bit-packed    */
/* planar lattice (X plane then Y plane, L rows of L/32 words, bit x%32 of   */
/* word x/32), for sizes where one byte per site would not fit in memory.    */
/* ------------------------------------------------------------------------ */
static inline int planar_bit(const uint32_t *plane, int64_t L, int64_t x, int64_t y) {
    return (int)((plane[y * (L / 32) + x / 32] >> (x % 32)) & 1u);
}

void oo_w2_sums_planar(int64_t L, const uint32_t *words, int64_t *s1, uint64_t *s2_lo,
                       uint64_t *s2_hi, int64_t *hmax) {
    const uint32_t *Xp = words, *Yp = words + L * (L / 32);
    i128 S1 = 0;
    u128 S2 = 0;
    int64_t hm = 0, h0 = 0;
    for (int64_t y = 0; y < L; ++y) {
        if (y > 0) h0 += 2 * (int64_t)planar_bit(Yp, L, 0, y) - 1;
        int64_t h = h0;
        for (int64_t x = 0; x < L; ++x) {
            if (x > 0) h += 2 * (int64_t)planar_bit(Xp, L, x, y) - 1;
            S1 += h;
            S2 += (u128)((i128)h * h);
            int64_t ah = h < 0 ? -h : h;
            if (ah > hm) hm = ah;
        }
    }
    *s1 = (int64_t)S1;
    *s2_lo = (uint64_t)S2;
    *s2_hi = (uint64_t)(S2 >> 64);
    if (hmax) *hmax = hm;
}

int oo_invariants_planar(int64_t L, const uint32_t *words, int64_t circ_y0, int64_t circ_y1) {
    const uint32_t *Xp = words, *Yp = words + L * (L / 32);
    int bad = 0;
    for (int64_t y = 0; y < L; ++y) {
        int64_t n = 0;
        for (int64_t x = 0; x < L; ++x) n += planar_bit(Xp, L, x, y);
        if (2 * n != L) bad |= 1;
    }
    int64_t *col = (int64_t *)calloc((size_t)L, sizeof(int64_t));
    if (!col) return -1;
    for (int64_t y = 0; y < L; ++y)
        for (int64_t x = 0; x < L; ++x) col[x] += planar_bit(Yp, L, x, y);
    for (int64_t x = 0; x < L; ++x)
        if (2 * col[x] != L) bad |= 2;
    free(col);
    for (int64_t y = circ_y0; y < circ_y1; ++y)
        for (int64_t x = 0; x < L; ++x) {
            const int64_t x1 = wrap(x + 1, L), y1 = wrap(y + 1, L);
            const int64_t circ = (2 * planar_bit(Xp, L, x1, y) - 1) + (2 * planar_bit(Yp, L, x1, y1) - 1) -
                                 (2 * planar_bit(Xp, L, x1, y1) - 1) - (2 * planar_bit(Yp, L, x, y1) - 1);
            if (circ != 0) bad |= 4;
        }
    return bad;
}
