// Two-time autocorrelation sums (Sec. 2: C(t,s) of Eq. (5) and its height and
// slope forms C_h, C_s) of a lattice at time t against a stored lattice at the
// waiting time s.
//
// Heights of each lattice are taken relative to its own h(0,0) = 0 (the
// covariance of two fields does not depend on a constant offset of either):
//   h(0,y) = sum_{y'=1..y} (2 Y(0,y') - 1),  h(x,y) = h(0,y) + r(x,y),
//   r(x,y) = sum_{x'=1..x} (2 X(x',y) - 1).
// Wanted: S_t = sum h_t, S_s = sum h_s, C = sum h_t h_s (128-bit), and the
// slope occupations sum X_t X_s, sum Y_t Y_s, sum (X_t + Y_t), sum (X_s + Y_s).
//
// Pass 1 (one warp per row, both lattices side by side): with q(x) the step
// sum over x' = 0..x and s0 the step of bit 0, r = q - s0, so
//   sum r_t r_s = sum q_t q_s - s0_s sum q_t - s0_t sum q_s + L s0_t s0_s.
// A warp takes the row in chunks of 256 words, 8 consecutive words per lane
// and plane (16-byte loads); inside a lane the running sums are built one
// nibble pair (four sites of both lattices) at a time from a 256-entry table
// (per pair: the sums of both nibbles' running steps, of their products, the
// net steps and the common up-slopes) and integer multiply-adds, and a packed
// warp scan of both lattices' step counts lifts the lane sums to the row.
// Pass 2: a scan of the column-0 Y bits gives h(0,y) of both lattices, and
// S_t, S_s and C accumulate in 64/128-bit integers, per block of rows and then
// over the blocks:
//   C = sum_y [L h0_t h0_s + h0_t R_s + h0_s R_t + R_ts].
// Row terms are at most L^3 in magnitude (2^60 at the largest L, 2^20).
#include "oct_internal.h"

namespace oct {
namespace {

constexpr uint32_t kFull = 0xFFFFFFFFu;
constexpr int kAcWarps = 8;

// Running steps of a nibble n (bit i = site i): a_i = sum_{j<=i} (2 b_j - 1).
__device__ __forceinline__ void nibble_steps(uint32_t n, int (&a)[4]) {
    int e = 0;
    for (int i = 0; i < 4; ++i) {
        e += ((n >> i) & 1u) ? 1 : -1;
        a[i] = e;
    }
}

// Table of the row pass, one entry per nibble pair e = n_t | n_s << 4 (four
// sites of lattice t and the same four of lattice s), with the running steps
// a_i of each nibble, t1 = sum a_i, n = a_3, X = sum a_i(t) a_i(s) and
// c = popcount(n_t & n_s):
//   .x = t1_s + (X + 30) 2^17 + 2^27 + n_s 2^28
//   .y = t1_t + c 2^17 + 2^27 + n_t 2^28          (mod 2^32)
// Read as signed words, floor(.x / 2^28) = n_s and floor(.y / 2^28) = n_t
// (the parts below bit 28 lie in [2^27 - 10, 2^28)).  Eight entries summed
// (a word) keep sum t1 + 2^16 in bits 0..16 (after adding 2^16) and
// sum (X + 30) <= 480, resp. sum c <= 32, in bits 17..25.
__device__ __forceinline__ uint2 pair_entry(uint32_t e) {
    int a[4], b[4];
    nibble_steps(e & 15u, a);
    nibble_steps(e >> 4, b);
    const int t1t = a[0] + a[1] + a[2] + a[3], t1s = b[0] + b[1] + b[2] + b[3];
    const int X = a[0] * b[0] + a[1] * b[1] + a[2] * b[2] + a[3] * b[3];
    const int c = __popc((e & 15u) & (e >> 4));
    uint2 r;
    r.x = static_cast<uint32_t>(t1s) + (static_cast<uint32_t>(X + 30) << 17) + (1u << 27) +
          (static_cast<uint32_t>(b[3]) << 28);
    r.y = static_cast<uint32_t>(t1t) + (static_cast<uint32_t>(c) << 17) + (1u << 27) +
          (static_cast<uint32_t>(a[3]) << 28);
    return r;
}

// hi32(a * b) + c, signed
__device__ __forceinline__ int ac_mad_hi(uint32_t a, int b, int c) {
    int d;
    asm("mad.hi.s32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(c));
    return d;
}

constexpr int kAcBlocksPerSM = 2;
constexpr int kAcLaneWords = 8;                      // words per lane, plane and chunk
constexpr uint32_t kAcChunkWords = 32u * kAcLaneWords;
constexpr int kAcTableBytes = 256 * 256;             // entry e of copy c at byte 256 e + 8 c

// Sums of one lane over the words of its chunk, relative to the lane's first
// site: Bt, Bs running steps before the current word, Lt = sum q_t,
// Ls = sum q_s, Lc = sum q_t q_s (all within 32 bits: |q| <= 256), and the
// counts nx (X_t & X_s), ny (Y_t & Y_s), yt, ys (Y bits).
struct AcLane {
    int Bt, Bs;
    int Lt, Ls, Lc;
    int nx, ny, yt, ys;
};

// One word pair: sites x..x+31 of X_t (wt) and X_s (ws).  With a_t, a_s the
// running steps inside the word and Pt_k, Ps_k those before nibble pair k
// (k = 0..7, in site order), the word adds
//   sum (Bt + a_t)(Bs + a_s) = 32 Bt Bs + Bt A_s + Bs A_t + C,
//   A = 4 sum P_k + sum t1,  C = sum (4 Pt Ps + Pt t1_s + Ps t1_t) + sum X.
// u = 4 Ps + .x is 4 Ps + t1_s in its low 17 bits (the fields above add
// multiples of 2^17), so two multiply-adds per pair give the first part of C
// exactly modulo 2^17 (|.| <= 7 * 3696 < 2^16); P advances by one
// multiply-high of each entry.
__device__ __forceinline__ void ac_word(const unsigned char *tab, uint32_t slot, uint32_t wt, uint32_t ws,
                                        AcLane &a) {
    // nibble pairs: z0 byte k = nibble 2k of both words, z1 byte k = nibble 2k + 1
    const uint32_t z0 = (wt & 0x0F0F0F0Fu) | ((ws << 4) & 0xF0F0F0F0u);
    const uint32_t z1 = ((wt >> 4) & 0x0F0F0F0Fu) | (ws & 0xF0F0F0F0u);
    uint2 e[8];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        e[2 * k] = *reinterpret_cast<const uint2 *>(tab + __byte_perm(z0, slot, 0x6504 + 16 * k));
        e[2 * k + 1] = *reinterpret_cast<const uint2 *>(tab + __byte_perm(z1, slot, 0x6504 + 16 * k));
    }
    int pt = ac_mad_hi(e[0].y, 16, 0), ps = ac_mad_hi(e[0].x, 16, 0);
    uint32_t acc = 0x10000u;
    int spt = 0, sps = 0;
#pragma unroll
    for (int k = 1; k < 8; ++k) {
        spt += pt;
        sps += ps;
        const uint32_t u = static_cast<uint32_t>(ps) * 4u + e[k].x;
        acc += static_cast<uint32_t>(pt) * u;
        acc += static_cast<uint32_t>(ps) * e[k].y;
        pt = ac_mad_hi(e[k].y, 16, pt);
        ps = ac_mad_hi(e[k].x, 16, ps);
    }
    uint32_t sx = 0x10000u, sy = 0x10000u;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        sx += e[k].x;
        sy += e[k].y;
    }
    const int At = 4 * spt + static_cast<int>(sy & 0x1FFFFu) - 0x10000;
    const int As = 4 * sps + static_cast<int>(sx & 0x1FFFFu) - 0x10000;
    const int C = static_cast<int>(acc & 0x1FFFFu) - 0x10000 + static_cast<int>((sx >> 17) & 0x1FFu) - 240;
    const int zs = 32 * a.Bs + As;
    a.Lt += 32 * a.Bt + At;
    a.Ls += zs;
    a.Lc += a.Bt * zs + a.Bs * At + C;
    a.nx += static_cast<int>((sy >> 17) & 0x3Fu);
    a.Bt += pt;
    a.Bs += ps;
}

// The lane's kAcLaneWords words of one plane at word w of a row (16-byte loads
// where the row allows them); words past the row's end read as 0.
__device__ __forceinline__ void ac_load(const uint32_t *row, uint32_t w, uint32_t wpr, bool vec_ok,
                                        uint32_t (&v)[kAcLaneWords]) {
    if (vec_ok && w + kAcLaneWords <= wpr) {
#pragma unroll
        for (int i = 0; i < kAcLaneWords / 4; ++i) {
            const uint4 q = *reinterpret_cast<const uint4 *>(row + w + 4 * i);
            v[4 * i] = q.x;
            v[4 * i + 1] = q.y;
            v[4 * i + 2] = q.z;
            v[4 * i + 3] = q.w;
        }
    } else {
#pragma unroll
        for (int i = 0; i < kAcLaneWords; ++i) v[i] = (w + i < wpr) ? row[w + i] : 0u;
    }
}

struct AcChunk {
    uint32_t xt[kAcLaneWords], xs[kAcLaneWords], yt[kAcLaneWords], ys[kAcLaneWords];
};

__device__ __forceinline__ void ac_load_chunk(const uint32_t *lt, const uint32_t *ls, size_t plane, size_t ro,
                                              uint32_t w, uint32_t wpr, bool vec_ok, AcChunk &ch) {
    ac_load(lt + ro, w, wpr, vec_ok, ch.xt);
    ac_load(ls + ro, w, wpr, vec_ok, ch.xs);
    ac_load(lt + plane + ro, w, wpr, vec_ok, ch.yt);
    ac_load(ls + plane + ro, w, wpr, vec_ok, ch.ys);
}

__global__ void __launch_bounds__(kAcWarps * 32, kAcBlocksPerSM)
    ac_rows_kernel(const uint32_t *lt, const uint32_t *ls, uint32_t L, AcRowSums *rows) {
    extern __shared__ __align__(16) unsigned char ac_table[];
    for (int i = threadIdx.x; i < 256; i += blockDim.x) {
        const uint2 e = pair_entry(static_cast<uint32_t>(i));
#pragma unroll
        for (int c = 0; c < 16; ++c) *reinterpret_cast<uint2 *>(ac_table + 256 * i + 8 * c) = e;
    }
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const uint32_t slot = 8u * static_cast<uint32_t>(lane & 15);
    const uint32_t wpr = L >> 5;
    const size_t plane = static_cast<size_t>(L) * wpr;
    const bool vec_ok = (wpr % 4u) == 0u && (reinterpret_cast<uintptr_t>(lt) % 16u) == 0u &&
                        (reinterpret_cast<uintptr_t>(ls) % 16u) == 0u;
    // The warp's rows y0, y0 + stride, ... chunk by chunk; the next chunk's
    // loads, across row ends too, are issued before the current one is reduced.
    const uint32_t stride = gridDim.x * kAcWarps;
    const uint32_t nchunks = (wpr + kAcChunkWords - 1) / kAcChunkWords;
    uint32_t y = blockIdx.x * kAcWarps + (threadIdx.x >> 5), c = 0;
    AcChunk cur, nxt;
    if (y < L) ac_load_chunk(lt, ls, plane, static_cast<size_t>(y) * wpr, kAcLaneWords * lane, wpr, vec_ok, cur);
    long long base_t = 0, base_s = 0;  // q just before the current chunk
    long long qt = 0, qs = 0, qts = 0;
    int nx = 0, ny = 0, mt = 0, ms = 0;
    while (y < L) {
        const uint32_t w0 = c * kAcChunkWords;
        const uint32_t w = w0 + kAcLaneWords * lane;
        const bool last = c + 1 == nchunks;
        const uint32_t ny_ = last ? y + stride : y, nc = last ? 0u : c + 1;
        if (ny_ < L)
            ac_load_chunk(lt, ls, plane, static_cast<size_t>(ny_) * wpr, nc * kAcChunkWords + kAcLaneWords * lane,
                          wpr, vec_ok, nxt);
        AcLane a{0, 0, 0, 0, 0, 0, 0, 0, 0};
        uint32_t nw = 0;
        if (w0 + kAcChunkWords <= wpr) {
#pragma unroll
            for (int j = 0; j < kAcLaneWords; ++j) {
                ac_word(ac_table, slot, cur.xt[j], cur.xs[j], a);
                a.ny += __popc(cur.yt[j] & cur.ys[j]);
                a.yt += __popc(cur.yt[j]);
                a.ys += __popc(cur.ys[j]);
            }
            nw = kAcLaneWords;
        } else {
#pragma unroll
            for (int j = 0; j < kAcLaneWords; ++j)
                if (w + j < wpr) {
                    ac_word(ac_table, slot, cur.xt[j], cur.xs[j], a);
                    a.ny += __popc(cur.yt[j] & cur.ys[j]);
                    a.yt += __popc(cur.yt[j]);
                    a.ys += __popc(cur.ys[j]);
                    ++nw;
                }
        }
        const int nbits = 32 * static_cast<int>(nw);
        // X popcounts from the net steps: popc = (net + bits) / 2
        mt += (a.Bt + nbits) / 2 + a.yt;
        ms += (a.Bs + nbits) / 2 + a.ys;
        nx += a.nx;
        ny += a.ny;
        // step counts of both lattices in one scan: |prefix| <= 8192 fits the
        // low 16 bits of a two's-complement packed word
        int incl = a.Bt + a.Bs * 65536;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int v = __shfl_up_sync(kFull, incl, o);
            if (lane >= o) incl += v;
        }
        const int incl_t = static_cast<short>(incl & 0xFFFF);
        const int incl_s = (incl - incl_t) / 65536;
        const int tot = __shfl_sync(kFull, incl, 31);
        const int tot_t = static_cast<short>(tot & 0xFFFF);
        const int tot_s = (tot - tot_t) / 65536;
        const long long Bt = base_t + (incl_t - a.Bt), Bs = base_s + (incl_s - a.Bs);
        qts += static_cast<long long>(nbits) * Bt * Bs + Bt * a.Ls + Bs * a.Lt + a.Lc;
        qt += static_cast<long long>(nbits) * Bt + a.Lt;
        qs += static_cast<long long>(nbits) * Bs + a.Ls;
        base_t += tot_t;
        base_s += tot_s;
        if (last) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                qt += __shfl_xor_sync(kFull, qt, o);
                qs += __shfl_xor_sync(kFull, qs, o);
                qts += __shfl_xor_sync(kFull, qts, o);
            }
            nx = __reduce_add_sync(kFull, nx);
            ny = __reduce_add_sync(kFull, ny);
            mt = __reduce_add_sync(kFull, mt);
            ms = __reduce_add_sync(kFull, ms);
            if (lane == 0) {
                const size_t ro = static_cast<size_t>(y) * wpr;
                const long long s0t = (lt[ro] & 1u) ? 1 : -1, s0s = (ls[ro] & 1u) ? 1 : -1;
                const long long Ll = L;
                AcRowSums o;
                o.rt = qt - Ll * s0t;
                o.rs = qs - Ll * s0s;
                o.rts = qts - s0s * qt - s0t * qs + Ll * s0t * s0s;
                o.ct = static_cast<int>(lt[plane + ro] & 1u);
                o.cs = static_cast<int>(ls[plane + ro] & 1u);
                o.nx = nx;
                o.ny = ny;
                o.mt = mt;
                o.ms = ms;
                rows[y] = o;
            }
            base_t = base_s = 0;
            qt = qs = qts = 0;
            nx = ny = mt = ms = 0;
        }
        y = ny_;
        c = nc;
        cur = nxt;
    }
}

// Pass 2 in two kernels, as for the roughness: pass 2a, one block per
// kAcBlockRows rows, sums relative to the heights of its first row
// (h0l = h0 - h0(first row), both lattices)
//   At = sum (L h0l_t + R_t),  As = sum (L h0l_s + R_s),
//   Cb = sum (L h0l_t h0l_s + h0l_t R_s + h0l_s R_t + R_ts),
// the occupation counts and the rises of h0l; it stores them over its first
// two row records (a block has at least 32 rows: L is a multiple of 32).
// Pass 2b scans the rises for the block heights H_t, H_s and adds
//   C = sum (Cb + H_t As + H_s At + L n H_t H_s),  S = sum (A + L n H).
constexpr int kAcBlockRows = 256;
constexpr int kAcCombineThreads = 1024;

struct AcBlockSums {
    long long at, as;
    unsigned long long c_lo;
    long long c_hi;      // Cb as a two's-complement 128-bit value
    long long nx, ny, mt, ms;
    int et, es;          // 2 h0l(last row) + Y(0, first row), per lattice
};
static_assert(sizeof(AcBlockSums) <= 2 * sizeof(AcRowSums), "a block record replaces two row records");

// 128-bit two's-complement sum of (lo, hi) pairs over a warp, in lane 0.
__device__ __forceinline__ void warp_sum_128(unsigned long long &lo, unsigned long long &hi) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long l2 = __shfl_down_sync(kFull, lo, o);
        const unsigned long long h2 = __shfl_down_sync(kFull, hi, o);
        const unsigned long long nl = lo + l2;
        hi = hi + h2 + (nl < lo ? 1ull : 0ull);
        lo = nl;
    }
}

__global__ void __launch_bounds__(kAcBlockRows) ac_block_kernel(AcRowSums *rows, uint32_t L) {
    __shared__ int wsum[kAcBlockRows / 32];
    __shared__ long long red[6][kAcBlockRows / 32];
    __shared__ unsigned long long clo[kAcBlockRows / 32], chi[kAcBlockRows / 32];
    __shared__ int last_t, last_s;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t y0 = blockIdx.x * kAcBlockRows;
    const uint32_t n = min(static_cast<uint32_t>(kAcBlockRows), L - y0);
    const bool valid = static_cast<uint32_t>(tid) < n;
    AcRowSums r{};
    if (valid) r = rows[y0 + tid];
    // column steps into row y of both lattices (none into the block's first
    // row), scanned together: |prefix| <= 256 fits the low 16 bits
    const int st = (valid && tid > 0) ? (r.ct ? 1 : -1) : 0, ss = (valid && tid > 0) ? (r.cs ? 1 : -1) : 0;
    int incl = st + ss * 65536;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int v = __shfl_up_sync(kFull, incl, o);
        if (lane >= o) incl += v;
    }
    if (lane == 31) wsum[warp] = incl;
    __syncthreads();
    for (int w = 0; w < warp; ++w) incl += wsum[w];
    const long long ht = static_cast<short>(incl & 0xFFFF);
    const long long hs = (incl - static_cast<int>(ht)) / 65536;
    if (static_cast<uint32_t>(tid) == n - 1) {
        last_t = static_cast<int>(ht);
        last_s = static_cast<int>(hs);
    }
    const long long Ll = L;
    long long v[6] = {0, 0, 0, 0, 0, 0};
    unsigned long long lo = 0, hi = 0;
    if (valid) {
        v[0] = Ll * ht + r.rt;
        v[1] = Ll * hs + r.rs;
        v[2] = r.nx;
        v[3] = r.ny;
        v[4] = r.mt;
        v[5] = r.ms;
        const __int128 c = static_cast<__int128>(Ll * ht * hs) + static_cast<__int128>(ht * r.rs) +
                           static_cast<__int128>(hs * r.rt) + static_cast<__int128>(r.rts);
        lo = static_cast<unsigned long long>(c);
        hi = static_cast<unsigned long long>(static_cast<unsigned __int128>(c) >> 64);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
        for (int i = 0; i < 6; ++i) v[i] += __shfl_down_sync(kFull, v[i], o);
    warp_sum_128(lo, hi);
    if (lane == 0) {
        for (int i = 0; i < 6; ++i) red[i][warp] = v[i];
        clo[warp] = lo;
        chi[warp] = hi;
    }
    __syncthreads();
    if (tid == 0) {
        AcBlockSums b{};
        long long a[6] = {0, 0, 0, 0, 0, 0};
        unsigned __int128 c = 0;
        for (int w = 0; w < kAcBlockRows / 32; ++w) {
            for (int i = 0; i < 6; ++i) a[i] += red[i][w];
            c += (static_cast<unsigned __int128>(chi[w]) << 64) | clo[w];
        }
        b.at = a[0];
        b.as = a[1];
        b.nx = a[2];
        b.ny = a[3];
        b.mt = a[4];
        b.ms = a[5];
        b.c_lo = static_cast<unsigned long long>(c);
        b.c_hi = static_cast<long long>(static_cast<unsigned long long>(c >> 64));
        b.et = 2 * last_t + r.ct;  // thread 0 holds the block's first row
        b.es = 2 * last_s + r.cs;
        *reinterpret_cast<AcBlockSums *>(rows + y0) = b;
    }
}

__global__ void __launch_bounds__(kAcCombineThreads)
    ac_combine_kernel(const AcRowSums *rows, uint32_t L, AcResult *out) {
    __shared__ long long part_t[kAcCombineThreads], part_s[kAcCombineThreads];
    __shared__ long long red[6][kAcCombineThreads / 32];
    __shared__ unsigned long long clo[kAcCombineThreads / 32], chi[kAcCombineThreads / 32];
    const int tid = threadIdx.x;
    const uint32_t nb = (L + kAcBlockRows - 1) / kAcBlockRows;
    const uint32_t per = (nb + kAcCombineThreads - 1) / kAcCombineThreads;
    const uint32_t b_begin = min(nb, tid * per), b_end = min(nb, (tid + 1) * per);
    auto rec = [&](uint32_t b) {
        return *reinterpret_cast<const AcBlockSums *>(rows + static_cast<size_t>(b) * kAcBlockRows);
    };
    // step into a block's first row (none into row 0) and rise to its last row
    auto step_in = [](int e, uint32_t b) { return b > 0 ? ((e & 1) ? 1ll : -1ll) : 0ll; };
    long long lt = 0, ls = 0;
    for (uint32_t b = b_begin; b < b_end; ++b) {
        const AcBlockSums r = rec(b);
        lt += step_in(r.et, b) + (r.et >> 1);
        ls += step_in(r.es, b) + (r.es >> 1);
    }
    part_t[tid] = lt;
    part_s[tid] = ls;
    __syncthreads();
    for (int o = 1; o < kAcCombineThreads; o <<= 1) {
        const long long vt = (tid >= o) ? part_t[tid - o] : 0;
        const long long vs = (tid >= o) ? part_s[tid - o] : 0;
        __syncthreads();
        part_t[tid] += vt;
        part_s[tid] += vs;
        __syncthreads();
    }
    long long last_t = part_t[tid] - lt, last_s = part_s[tid] - ls;  // h0 of the last row before b_begin
    const long long Ll = L;
    long long v[6] = {0, 0, 0, 0, 0, 0};
    __int128 C = 0;
    for (uint32_t b = b_begin; b < b_end; ++b) {
        const AcBlockSums r = rec(b);
        const long long Ht = last_t + step_in(r.et, b), Hs = last_s + step_in(r.es, b);
        const long long nr = min(static_cast<uint32_t>(kAcBlockRows), L - b * kAcBlockRows);
        const __int128 Cb = static_cast<__int128>((static_cast<unsigned __int128>(r.c_hi) << 64) | r.c_lo);
        C += Cb + static_cast<__int128>(Ht) * r.as + static_cast<__int128>(Hs) * r.at +
             static_cast<__int128>(Ll * nr) * Ht * Hs;
        v[0] += r.at + Ll * nr * Ht;
        v[1] += r.as + Ll * nr * Hs;
        v[2] += r.nx;
        v[3] += r.ny;
        v[4] += r.mt;
        v[5] += r.ms;
        last_t = Ht + (r.et >> 1);
        last_s = Hs + (r.es >> 1);
    }
    // block reduction; C as a two's-complement 128-bit value in (lo, hi)
    unsigned long long lo = static_cast<unsigned long long>(C);
    unsigned long long hi = static_cast<unsigned long long>(static_cast<unsigned __int128>(C) >> 64);
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
        for (int i = 0; i < 6; ++i) v[i] += __shfl_down_sync(kFull, v[i], o);
    warp_sum_128(lo, hi);
    if ((tid & 31) == 0) {
        for (int i = 0; i < 6; ++i) red[i][tid >> 5] = v[i];
        clo[tid >> 5] = lo;
        chi[tid >> 5] = hi;
    }
    __syncthreads();
    if (tid == 0) {
        long long a[6] = {0, 0, 0, 0, 0, 0};
        unsigned __int128 c = 0;
        for (int w = 0; w < kAcCombineThreads / 32; ++w) {
            for (int i = 0; i < 6; ++i) a[i] += red[i][w];
            c += (static_cast<unsigned __int128>(chi[w]) << 64) | clo[w];
        }
        out->sum_ht = a[0];
        out->sum_hs = a[1];
        out->occ_x = a[2];
        out->occ_y = a[3];
        out->m_t = a[4];
        out->m_s = a[5];
        out->cross_lo = static_cast<unsigned long long>(c);
        out->cross_hi = static_cast<unsigned long long>(c >> 64);
    }
}

}  // namespace

cudaError_t launch_two_time(const uint32_t *lat_t, const uint32_t *lat_s, uint32_t L, AcRowSums *rows,
                            AcResult *out, cudaStream_t st) {
    // one wave of resident blocks (64 KB of table each), rows taken grid-stride;
    // the table needs the dynamic shared-memory limit raised once per device
    constexpr int kMaxDevices = 64;
    static int sms[kMaxDevices] = {};
    static bool smem_set[kMaxDevices] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    if (sms[dev] <= 0) {
        e = cudaDeviceGetAttribute(&sms[dev], cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return e;
    }
    if (!smem_set[dev]) {
        e = cudaFuncSetAttribute(ac_rows_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kAcTableBytes);
        if (e != cudaSuccess) return e;
        smem_set[dev] = true;
    }
    const uint64_t want = (static_cast<uint64_t>(L) + kAcWarps - 1) / kAcWarps;
    const uint64_t wave = static_cast<uint64_t>(sms[dev]) * kAcBlocksPerSM;
    const int blocks = static_cast<int>(want < wave ? want : wave);
    ac_rows_kernel<<<blocks, kAcWarps * 32, kAcTableBytes, st>>>(lat_t, lat_s, L, rows);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    ac_block_kernel<<<(L + kAcBlockRows - 1) / kAcBlockRows, kAcBlockRows, 0, st>>>(rows, L);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    ac_combine_kernel<<<1, kAcCombineThreads, 0, st>>>(rows, L, out);
    return cudaGetLastError();
}

}  // namespace oct
