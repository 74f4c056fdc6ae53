/*
 * oct.h -- C ABI of the GB300 octahedron-model DTrDT simulator.
 *
 * The library simulates random-sequential (RS) updating of the 2+1-d
 * octahedron model for KPZ surface growth (Kelling, Odor, Gemming,
 * "Suppressing correlations in massively parallel simulations of lattice
 * models", arXiv:1705.01022) under the DTrDT domain decomposition: double
 * tiling with a random origin at device level (Sec. 3, "DTr"), single-hit
 * double tiling at block level (Sec. 3.1).  The roughness W^2 of Eq. (3) is
 * measured exactly.
 *
 * Conventions shared by every entry point:
 *   - All functions return an oct error code (OCT_OK = 0).  No C++ exception
 *     crosses this boundary.  oct_last_error() gives a message for the most
 *     recent failure on the calling thread.
 *   - A handle may be used by one host thread at a time.
 *   - Work is enqueued on the handle's CUDA stream (the caller's, if one was
 *     given to oct_create_ex, else one the library creates).  Functions that
 *     return data to the host synchronise that stream; oct_run_mcs does not.
 *   - Device pointers and streams are plain void* (cudaStream_t / device
 *     addresses) so that no CUDA or PyTorch type appears in the ABI.
 *
 * Lattice layouts.
 *   Slope bits (Sec. 2.1, Eq. (1); on-site convention of Sec. 3): for site
 *   (x, y), X = 1 iff h(x,y) - h(x-1,y) = +1 and Y = 1 iff
 *   h(x,y) - h(x,y-1) = +1, indices periodic in L.
 *   - Canonical layout (the paper's data structure: one 32-bit word holds
 *     4x4 sites, Sec. 3.1): L*L/16 words; word (y/4)*(L/4) + x/4 holds
 *     X at bit 2*(4*(y%4) + x%4) and Y at the next bit.
 *   - Planar layout (device-resident form): an X plane then a Y plane, each L
 *     rows of L/32 words; bit i of word w of row y is the slope bit of site
 *     (32w + i, y).  Both layouts occupy L*L/4 bytes.
 */
#ifndef OCT_H
#define OCT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Error codes. */
#define OCT_OK 0
#define OCT_EINVAL 1       /* invalid argument (sizes, probabilities, layout)      */
#define OCT_ENOMEM 2       /* device or host allocation failed                     */
#define OCT_ECUDA 3        /* a CUDA runtime call failed                           */
#define OCT_ETIMEDOUT 4    /* a bounded device wait gave up                        */
#define OCT_EINTERNAL 5    /* an internal consistency check failed                 */
#define OCT_EUNSUPPORTED 6 /* valid request the library does not implement       */

typedef struct oct_sim oct_sim; /* opaque; owns its device memory unless told otherwise */

/* Creation parameters (oct_create_ex).  Zero fields take the defaults.
 *   L      lateral size; needs L % (2*Bx) == 0 and L % (2*By) == 0.
 *   p, q   deposition / removal probabilities of Eq. (1), each in [0, 1].
 *   seed   Philox-4x32-10 key (low word, high word).
 *   Bx, By device-layer sub-tile in sites (device tile 2Bx x 2By).  Bx must be
 *          a multiple of 32 and By a multiple of 4*cy; a sub-tile may hold at
 *          most 32 groups of 32 x 4cy sites.  Defaults: 64 x 64 if L % 128 == 0,
 *          else 32 x 16.
 *   cx, cy block-layer thread cell in sites (default 4 x 4, the one cell
 *          shape the library implements; others give OCT_EUNSUPPORTED).
 *   stream cudaStream_t to enqueue on, or NULL for a library-owned stream
 *          (pass cudaStreamLegacy, 0x1, for the legacy default stream).
 *   lattice  external device buffer of L*L/4 bytes (planar layout), or NULL
 *          for a library-owned one.  An external buffer stays owned by the
 *          caller and must outlive the handle.
 *   no_init  0: write the flat start h = (x+y) mod 2; 1: keep the buffer.
 *   scheme   block-layer decomposition (Sec. 3.1): OCT_SCHEME_DT (default,
 *          DTrDT: single-hit double tiling), OCT_SCHEME_DB (DTrDB:
 *          single-hit dead border; border attempts are delayed after the bulk
 *          ones when both p and q are non-zero, otherwise all attempts of a
 *          step are carried out together, as in the paper's runs) or
 *          OCT_SCHEME_DTR (DTrDTr, Sec. 4.1.2: single-hit double tiling whose
 *          block-layer origin moves to a uniform position in the thread cell
 *          after every collective step, the cell grid wrapping around the
 *          sub-tile). */
#define OCT_SCHEME_DT 0
#define OCT_SCHEME_DB 1
#define OCT_SCHEME_DTR 2
typedef struct {
    int64_t L;
    double p, q;
    uint64_t seed;
    int32_t Bx, By;
    int32_t cx, cy;
    void *stream;
    void *lattice;
    int32_t no_init;
    int32_t scheme;
    /* Row strip of a lattice split over several devices (strip_rows = 0: the
     * handle holds the whole lattice).  The handle's buffer then holds
     * held_rows full rows from global row strip_row0 on (planar: held_rows
     * rows of X, then held_rows rows of Y; held_rows * L / 4 bytes), and its
     * device steps update the device-tile rows whose first row lies in
     * [strip_row0, strip_row0 + strip_rows).  strip_row0 and strip_rows must be
     * multiples of 2*By, held_rows >= strip_rows + 2*By and <= L. */
    int32_t strip_row0, strip_rows, held_rows;
    int32_t reserved[3];
} oct_params;

/* Exact roughness, Eq. (3), read as the mean over all L^2 sites:
 *   heights relative to h(0,0) = 0, s1 = sum h, s2 = sum h^2 as an unsigned
 *   128-bit value (s2_hi:s2_lo), w2 = (N*s2 - s1^2) / N^2 with N = n_sites,
 *   formed in 128-bit integers and converted to double once.
 *   net_flips = accepted depositions minus removals since the flat start
 *   (the absolute mean height grows by 2*net_flips/N); hmax = max |h|. */
typedef struct {
    int64_t t;
    int64_t n_sites;
    int64_t s1;
    uint64_t s2_lo, s2_hi;
    int64_t net_flips;
    int64_t hmax;
    double w2;
} oct_w2;

typedef struct {
    int64_t L;
    int64_t t;
    int32_t Bx, By, cx, cy;
    double p, q;
    uint64_t seed;
    void *stream;
    void *lattice; /* device address of the planar lattice */
    int64_t lattice_bytes;
    int32_t scheme;
    int32_t reserved;
} oct_info;

/* Creates a simulation in the flat start with the default tiling (see
 * oct_params).  *out receives the handle.  Errors: OCT_EINVAL (L, p, q),
 * OCT_ENOMEM, OCT_ECUDA. */
int oct_create(int64_t L, double p, double q, uint64_t seed, oct_sim **out);

/* Creates a simulation from a parameter block (see oct_params). */
int oct_create_ex(const oct_params *prm, oct_sim **out);

/* Enqueues n >= 0 Monte Carlo steps (one MCS = one sweep of L^2 update
 * attempts, Sec. 2.1) and advances the handle's time t by n.  Each MCS draws
 * a new random origin and set order (DTr, Sec. 3) and runs four device steps
 * of single-hit DT on every sub-tile of one set (Sec. 3.1).  Asynchronous on
 * the handle's stream.  Errors: OCT_EINVAL (n < 0 or t would pass 2^32-1). */
int oct_run_mcs(oct_sim *s, int64_t n);

/* One device step at a time (for a lattice split into row strips over several
 * devices, whose halo rows are exchanged between device steps).
 * oct_device_step enqueues device step k (0..3, in this order) of the current
 * MCS: the sub-tiles of set perm[k] (Sec. 3, DTr); oct_end_mcs then advances
 * t by one.  Four device steps and oct_end_mcs equal oct_run_mcs(s, 1).
 * Errors: OCT_EINVAL (k outside 0..3, t would pass 2^32-1). */
int oct_device_step(oct_sim *s, int k);
int oct_end_mcs(oct_sim *s);

/* The device layer's draw of MCS t for a lattice of side L under `seed`
 * (Sec. 3, DTr), computed on the host exactly as the kernels do: the origin
 * (ox, oy) and the order perm[0..3] of the four sub-tile sets (set sigma is
 * quadrant (sigma & 1, sigma >> 1) of every device tile).  Strip exchanges
 * need it: after device step k of a strip, the rows of the next strip it has
 * changed are its first ((oy - strip_row0) mod 2By) + By*(perm[k] >> 1) -
 * By + 1 (none if that is <= 0). */
int oct_mcs_draw(uint64_t seed, int64_t L, uint32_t t, int64_t *ox, int64_t *oy, int32_t perm[4]);

/* Exact roughness of a lattice split into row strips (Eq. (3)).  For its own
 * rows (buffer rows 0 .. strip_rows-1) a strip handle reports, with heights
 * e_j + r(x) relative to its first row's h(0, .) (e_j = sum over its rows
 * 1..j of 2 Y(0,.) - 1, r as for W^2):
 *   rows, L, f = 2 Y(0, first row) - 1, e_last = e of its last row,
 *   p1 = sum (e_j + r), p2 = sum (e_j + r)^2 (128-bit, non-negative),
 *   lo = min (e_j + r), hi = max (e_j + r), net_flips.
 * oct_strip_combine takes the strips of one lattice in row order (their rows
 * must add up to L) and forms S1, S2, hmax and W^2 exactly: the first row of
 * strip r stands at B_r = B_{r-1} + e_last_{r-1} + f_r (B_0 = 0), so its rows
 * add L rows B_r + p1 to S1 and L rows B_r^2 + 2 B_r p1 + p2 to S2.
 * oct_strip_measure synchronises the handle's stream. */
typedef struct {
    int64_t rows, L;
    int64_t f, e_last;
    int64_t p1;
    uint64_t p2_lo, p2_hi;
    int64_t lo, hi;
    int64_t t, net_flips;
} oct_strip_sums;
int oct_strip_measure(oct_sim *s, oct_strip_sums *out);
int oct_strip_combine(const oct_strip_sums *parts, int64_t n, oct_w2 *out);

/* Computes the exact roughness of the current lattice (Eq. (3)); synchronises
 * the handle's stream.  OCT_EINVAL while an asynchronous measurement of the
 * handle is pending. */
int oct_measure_w2(oct_sim *s, oct_w2 *out);

/* The same measurement in two halves, so that one host thread can keep
 * several handles busy.  oct_measure_w2_async enqueues the reduction and the
 * read-back of its sums on the handle's stream and returns at once; it
 * measures the lattice as it stands after the work enqueued before it (later
 * oct_run_mcs calls do not change the result).  oct_w2_wait synchronises the
 * handle's stream and fills *out (out->t is the time of the measured lattice).
 * One measurement may be pending per handle: a second oct_measure_w2_async, or
 * oct_measure_w2, before oct_w2_wait returns OCT_EINVAL, and so does
 * oct_w2_wait with nothing pending. */
int oct_measure_w2_async(oct_sim *s);
int oct_w2_wait(oct_sim *s, oct_w2 *out);

/* Copies the lattice to host memory in the canonical 4x4-per-word layout;
 * words must equal L*L/16.  Synchronises. */
int oct_get_lattice(oct_sim *s, uint32_t *host, size_t words);

/* Replaces the lattice from host memory (canonical layout, words = L*L/16)
 * and sets the time to t (resume from a snapshot: the counter-based random
 * streams make the continuation identical to an uninterrupted run).  The
 * caller is responsible for the lattice being a valid slope field; the
 * accumulated net-flip count is reset to 0. */
int oct_set_lattice(oct_sim *s, const uint32_t *host, size_t words, int64_t t);

/* Raw copies of the planar layout (words = L*L/16 in total: X plane then Y
 * plane).  oct_get_planes and oct_set_planes synchronise the handle's stream
 * (oct_set_planes also sets the time to t and restarts the flip counters). */
int oct_get_planes(oct_sim *s, uint32_t *host, size_t words);
int oct_set_planes(oct_sim *s, const uint32_t *host, size_t words, int64_t t);

/* Enqueues the copy of both planes to `host` on the handle's stream and
 * returns at once.  The data is there after the next synchronising call on
 * the handle (oct_sync, oct_w2_wait, ...); until then the caller keeps `host`
 * alive and does not read it.  With page-locked `host` the copy overlaps other
 * handles' kernels and host-to-device copies. */
int oct_get_planes_async(oct_sim *s, uint32_t *host, size_t words);

/* Copies a W x H window whose corner is global site (wx, wy) (periodic) into
 * host byte arrays X, Y of W*H entries each (index j*W + i for site
 * (wx+i, wy+j)), one slope bit per byte.  Synchronises. */
int oct_get_window(oct_sim *s, int64_t wx, int64_t wy, int64_t W, int64_t H, uint8_t *X,
                   uint8_t *Y);

/* Parameters and current time of a handle. */
int oct_get_info(oct_sim *s, oct_info *out);

/* Waits for all work enqueued on the handle's stream. */
int oct_sync(oct_sim *s);

/* Per-kernel device time (milliseconds) accumulated while timing is on:
 * step_ms covers the device-step kernels (MCS draw, staging, single-hit
 * steps, flip counting), other_ms the rest of oct_run_mcs.  Timing brackets every device-step launch with CUDA events on
 * the handle's stream.  oct_set_timing(s, 1) enables and resets the
 * counters. */
int oct_set_timing(oct_sim *s, int enable);
int oct_get_timing(oct_sim *s, double *step_ms, int64_t *step_launches, double *other_ms);

/* Counters since the flat start or the last oct_set_lattice/oct_set_planes:
 * net_flips = accepted depositions minus removals, draws = attempts that
 * landed on an eligible site whose probability lies strictly in (0,1) and so
 * needed an acceptance draw (counted only when p or q lies strictly inside
 * (0,1)), tail_blocks = Philox blocks the plain device-step kernels generated
 * for the tail stream of tied acceptance uniforms (counted over the lanes that
 * store them; zero without acceptance draws).  Synchronises. */
typedef struct {
    int64_t t;
    int64_t net_flips;
    int64_t draws;
    int64_t tail_blocks;  /* Philox-4x32-10 blocks generated for the tail stream
                             of tied acceptance uniforms (128 random bits each) */
} oct_stats;
int oct_get_stats(oct_sim *s, oct_stats *out);

/* Measures the integer-pipe throughput of the current device: op 0 runs
 * chains of three-input logic (LOP3), op 1 of 32-bit multiply-add (IMAD), on
 * every SM.  Returns operations per SM per clock, the SM clock seen during the
 * probe (from the SM cycle counter over the kernel's event time) and the SM
 * count.  Used as the denominator of the hot path's integer roofline; the
 * paper has no counterpart. */
int oct_probe_int_rate(int op, double *ops_per_clk_per_sm, double *sm_mhz, int *sm_count);

/* Exact roughness of a lattice the caller owns, without allocating memory.
 * (The paper has no counterpart; this serves callers that cannot allocate.)
 * For callers such as a plugin or framework that owns all device memory and
 * hands over only a buffer and a stream, or a latency-critical loop where
 * cudaMalloc/cudaFree are not allowed because they may synchronise the
 * device.  It computes what oct_measure_w2 computes (the same sums, the same
 * W^2) for the planar lattice at device address `lattice` (L*L/4 bytes,
 * 16-byte aligned), enqueued on `stream` (a cudaStream_t, NULL for the
 * default stream), then synchronises that stream and writes out->s1, s2,
 * hmax, n_sites and w2 (out->t = -1 and out->net_flips = 0: a bare lattice
 * carries neither).  Scratch lives in one fixed device array of 4 MiB + 256
 * bytes compiled into the library, which every GPU that loads the library
 * holds until the process exits; it serves L up to 131072 (2^17) and larger L
 * is rejected with OCT_EINVAL and a message in oct_last_error().  The first
 * call on each device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current and keeps it for the rest
 * of the process; make that first call before any stream capture.  The kept
 * address belongs to the device's context at that first call and does not
 * survive a cudaDeviceReset: do not use this entry point on a device that was
 * reset earlier in the same process.  All calls share the one array: calls
 * that may overlap on the GPU (other streams, other threads) race and must be
 * serialised by the caller.  It calls no cudaMalloc, cudaFree or other
 * allocating routine. */
int oct_w2_noalloc(const void *lattice, int64_t L, void *stream, oct_w2 *out);

/* ---------------------------------------------------------------------------
 * Two-time autocorrelations (Sec. 2: C(t,s) of Eq. (5) and its forms for the
 * slopes, C_s, and the heights, C_h).  The paper writes the height form with
 * squared heights; its own identity C_h(s,s) = W^2(s) fixes the product of the
 * heights at the two times, which is what is computed here.  <.> is the mean
 * over the sites of one sample (averaging over samples is the caller's):
 *   C_h(t,s) = <h(t) h(s)> - <h(t)><h(s)>
 *            = (N*cross - sum_ht*sum_hs) / N^2,            N = L*L,
 *   C_s(t,s) = <n(t) n(s)> - <n(t)><n(s)> over the 2N lattice-gas variables
 *            n = X and n = Y (the slope bits of Eq. (1))
 *            = (2N*(occ_x + occ_y) - m_t*m_s) / (2N)^2.
 * Heights of each lattice are relative to its own h(0,0) = 0: C_h does not
 * depend on a constant offset of either field.  Numerators are formed in
 * 128-bit integers and converted to double once; at t = s, c_h equals the w2
 * of oct_measure_w2 exactly and c_s = 1/4 on any valid slope field.
 * ------------------------------------------------------------------------- */
typedef struct {
    int64_t t;          /* time of the current lattice (MCS); -1 from oct_two_time_planes */
    int64_t s;          /* waiting time: time of the snapshot (MCS); -1 likewise */
    int64_t n_sites;    /* N = L*L */
    int64_t sum_ht;     /* sum over sites of h(t) */
    int64_t sum_hs;     /* sum over sites of h(s) */
    uint64_t cross_lo;  /* sum over sites of h(t) h(s): low 64 bits of a signed 128-bit value */
    int64_t cross_hi;   /* its high 64 bits (two's complement) */
    int64_t occ_x;      /* sum of X_t X_s (x slope up at both times) */
    int64_t occ_y;      /* sum of Y_t Y_s */
    int64_t m_t;        /* sum of X_t + Y_t */
    int64_t m_s;        /* sum of X_s + Y_s */
    double c_h;         /* C_h(t,s) */
    double c_s;         /* C_s(t,s) */
    int64_t reserved[4];
} oct_ac;

/* Stores a device copy of the current lattice as the state at the waiting
 * time s = the handle's current t (L*L/4 bytes, allocated on the first call
 * and owned by the handle; a later call overwrites it).  Asynchronous on the
 * handle's stream. */
int oct_snapshot(oct_sim *s);

/* C_h(t,s) and C_s(t,s) of the current lattice (time t) against the last
 * snapshot (time s).  Synchronises the handle's stream.  Errors: OCT_EINVAL if
 * no snapshot was taken. */
int oct_measure_ac(oct_sim *s, oct_ac *out);

/* The same for two planar device lattices the caller owns (X plane then Y
 * plane, L*L/4 bytes each; 16-byte aligned buffers take the vector path),
 * e.g. a batched replica and a copy of it.  L even, a multiple of 32, at most
 * 2^20.  Enqueued on `stream` (NULL: the legacy default stream) with
 * stream-ordered scratch (cudaMallocAsync of about 48*L bytes), then
 * synchronises the stream.  out->t = out->s = -1. */
int oct_two_time_planes(const void *lat_t, const void *lat_s, int64_t L, void *stream, oct_ac *out);

/* ---------------------------------------------------------------------------
 * Batched replicas.  Many independent realizations (each its own L, p, q and
 * key; every one the same DTrDT dynamics as a single handle, bit for bit) are
 * advanced together: every device step of every replica runs in one launch
 * per acceptance mode, and one MCS is captured once in a CUDA graph and
 * replayed.  Replica lattices are device-resident, planar layout.
 * ------------------------------------------------------------------------- */
typedef struct oct_batch oct_batch;

/* One replica: L a multiple of 64 in [64, 16384]; p, q in [0, 1]; seed its
 * Philox key; Bx, By its sub-tile (0, 0: 64 x 64 if L % 128 == 0, else
 * 32 x 32).  The sub-tile must hold a power-of-two number of 32 x 16-site
 * groups in each direction, at most 32 in all. */
typedef struct {
    int64_t L;
    double p, q;
    uint64_t seed;
    int32_t Bx, By;
    int32_t reserved[6];
} oct_replica;

/* Key of replica r under a master seed: the first two words of
 * Philox-4x32-10 at counter (r, 0, 0, 6 << 28) under the master key. */
int oct_replica_seed(uint64_t master_seed, uint32_t r, uint64_t *seed);

/* Creates a batch holding n >= 0 replicas in the flat start, in slots
 * 0..n-1, on `stream` (NULL: library-owned).  Replica lattices come from a
 * stream-ordered memory pool private to the batch. */
int oct_batch_create(int64_t n, const oct_replica *reps, void *stream, oct_batch **out);

/* Adds one replica in the flat start at its own time t = 0 (continuous
 * batching: replicas may join while others are running); *slot receives its
 * slot index (a freed slot is reused).  Errors: OCT_EINVAL, OCT_ENOMEM. */
int oct_batch_add(oct_batch *b, const oct_replica *r, int64_t *slot);

/* Removes the replica in `slot` and returns its lattice to the pool. */
int oct_batch_remove(oct_batch *b, int64_t slot);

/* Enqueues n MCS for every replica in the batch (asynchronous); each replica
 * advances its own time t.  The work list and graph are rebuilt first if
 * replicas were added or removed; the rebuild copies the new work list in
 * stream order and does not wait for the device. */
int oct_batch_run(oct_batch *b, int64_t n);

/* Exact roughness of every slot (out holds one entry per slot index handed
 * out so far; free slots read as zeros; t is each replica's own time,
 * net_flips since its flat start).  Synchronises. */
int oct_batch_measure_w2(oct_batch *b, oct_w2 *out, int64_t n);

/* Exact roughness of the replica in one slot.  Synchronises. */
int oct_batch_measure_slot(oct_batch *b, int64_t slot, oct_w2 *out);

/* The same measurement without waiting: oct_batch_measure_async enqueues the
 * roughness reduction of the replica in `slot` as it stands at this point of
 * the batch's stream (after the MCS enqueued so far) and returns a ticket at
 * once; oct_batch_poll reports whether it is done (*ready = 1, *out filled) or
 * not yet (*ready = 0); oct_batch_wait blocks until it is.  The replica may be
 * removed (and its slot reused) right after the call: the measurement reads
 * the lattice before the removal takes effect.  The last 1024 tickets stay
 * valid; an older one is refused with OCT_EINVAL.  Serving streams W^2 back
 * this way without stalling the device (Sec. 2.1, Eq. (3); the scheduling is
 * this library's, the paper has no counterpart). */
int oct_batch_measure_async(oct_batch *b, int64_t slot, int64_t *ticket);
int oct_batch_poll(oct_batch *b, int64_t ticket, oct_w2 *out, int *ready);
int oct_batch_wait(oct_batch *b, int64_t ticket, oct_w2 *out);

/* Planar lattice of the replica in `slot` (words = L*L/16).  Synchronises. */
int oct_batch_get_planes(oct_batch *b, int64_t slot, uint32_t *host, size_t words);

/* Two-time autocorrelations of one replica (Sec. 2, Eq. (5); the same sums and
 * readings as oct_snapshot / oct_measure_ac).  oct_batch_snapshot stores the
 * replica's current lattice as its state at the waiting time s (its own MCS
 * count), in a buffer from the batch's memory pool that lives until the
 * replica is removed; a later call replaces it.  oct_batch_measure_ac reduces
 * the replica's current lattice against that snapshot; OCT_EINVAL without a
 * snapshot or for a free slot.  Both synchronise the batch's stream. */
int oct_batch_snapshot(oct_batch *b, int64_t slot);
int oct_batch_measure_ac(oct_batch *b, int64_t slot, oct_ac *out);

/* MCS run by oct_batch_run so far, replicas present, their total sites, and
 * their acceptance draws. */
int oct_batch_get_stats(oct_batch *b, int64_t *ticks, int64_t *n_active, int64_t *active_sites,
                        int64_t *draws);

/* Waits for the batch's stream. */
int oct_batch_sync(oct_batch *b);

/* Stream marks, so that a caller can bound how much work it keeps enqueued
 * ahead of the device (a serving loop that lets newly admitted replicas join
 * the next launches instead of queueing behind work already enqueued).
 * oct_batch_mark records the point the batch's stream has reached (after all
 * work enqueued so far) and returns its number in *mark; oct_batch_mark_done
 * sets *done = 1 once the device has passed it, else 0; oct_batch_mark_wait
 * blocks until it has.  The last 64 marks are kept: recording a new mark first
 * waits for the one 64 marks older, so an older mark always reads as passed.
 * Marks are this library's scheduling aid; the paper has no counterpart.
 * Errors: OCT_EINVAL for a NULL argument or a mark not handed out,
 * OCT_ECUDA. */
int oct_batch_mark(oct_batch *b, int64_t *mark);
int oct_batch_mark_done(oct_batch *b, int64_t mark, int *done);
int oct_batch_mark_wait(oct_batch *b, int64_t mark);

/* With timing on, oct_batch_run launches device step by device step (no
 * graph) and brackets each with CUDA events; step_ms sums them. */
int oct_batch_set_timing(oct_batch *b, int enable);
int oct_batch_get_timing(oct_batch *b, double *step_ms, int64_t *step_launches);

/* Releases the batch.  NULL-safe. */
int oct_batch_destroy(oct_batch *b);

/* Releases the handle and the memory it owns.  NULL-safe. */
int oct_destroy(oct_sim *s);

/* Static text for an error code. */
const char *oct_strerror(int code);

/* Message describing the most recent failure on this thread ("" if none). */
const char *oct_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* OCT_H */
