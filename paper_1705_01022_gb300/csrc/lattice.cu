// Lattice-wide kernels: flat start, exact roughness, layout conversion.
//
// Roughness (Eq. (3), mean over the L^2 sites): heights relative to h(0,0)=0,
//   h(0,y) = sum_{y'=1..y} (2 Y(0,y') - 1),
//   h(x,y) = h(0,y) + r(x,y),  r(x,y) = sum_{x'=1..x} (2 X(x',y) - 1).
// Pass 1 (one warp per row): with q(x) = sum_{x'=0..x} (2X(x',y)-1) and
// s0 = 2X(0,y)-1, r = q - s0, so the row sums of r and r^2 follow from those
// of q.  A warp takes the row in chunks of 512 words, 16 consecutive words per
// lane (16-byte coalesced loads); each lane reduces its words with a 256-entry
// byte table (per byte: the sum of the running step inside it, of its square,
// the net step and the extremes) and integer multiply-adds, and a warp scan of
// the lanes' net steps lifts the lane sums to the row.  Pass 2: a scan of the
// column bits gives h0 = h(0,y), and S1 = sum_y (L h0 + R1), S2 = sum_y (L h0^2 +
// 2 h0 R1 + R2) accumulate in 128-bit integers, per block of rows and then
// over the blocks.  Per-row terms are bounded by
// 4 L^3 < 2^63 for L <= 2^20, so only the cross-row sums need 128 bits.
#include "oct_internal.h"

namespace oct {
namespace {

constexpr uint32_t kFull = 0xFFFFFFFFu;

__global__ void init_flat_kernel(uint32_t *lat, uint32_t rows, uint64_t n_words, uint32_t wpr) {
    // X = Y = (x+y) & 1: odd x set on even rows, even x set on odd rows (the
    // buffer's first row is an even lattice row).
    for (uint64_t i = blockIdx.x * static_cast<uint64_t>(blockDim.x) + threadIdx.x; i < n_words;
         i += static_cast<uint64_t>(gridDim.x) * blockDim.x) {
        const uint64_t row = (i / wpr) % rows;
        lat[i] = (row & 1u) ? 0x55555555u : 0xAAAAAAAAu;
    }
}

// Byte table of the row pass.  For byte value v, with the running step
// e_i = sum_{j<=i} (2 b_j - 1), i = 0..7, t1 = sum e_i, t2 = sum e_i^2, n = e_7:
//   .x = 2 t1 + t2 2^17 + n 2^27   (mod 2^32; |2 t1| <= 72 < 2^17 <= t2 2^17)
//   .y = (min e_i + kW2Bias) | (kW2Bias - max e_i) << 16
// The four .x of a word plus 512 hold sum 2 t1 + 512 in bits 0..16 and
// sum t2 <= 816 in bits 17..26; read as a signed word, floor(.x / 2^27) = n
// (t2 >= 4, so the part below bit 27 is positive).
constexpr uint32_t kW2Bias = 0x8000u;

__device__ __forceinline__ uint2 byte_entry(uint32_t v) {
    int e = 0, s1 = 0, s2 = 0, mn = 1 << 20, mx = -(1 << 20);
    for (int i = 0; i < 8; ++i) {
        e += ((v >> i) & 1u) ? 1 : -1;
        s1 += e;
        s2 += e * e;
        mn = min(mn, e);
        mx = max(mx, e);
    }
    uint2 r;
    r.x = static_cast<uint32_t>(2 * s1) + (static_cast<uint32_t>(s2) << 17) + (static_cast<uint32_t>(e) << 27);
    r.y = (kW2Bias + static_cast<uint32_t>(mn)) | ((kW2Bias - static_cast<uint32_t>(mx)) << 16);
    return r;
}

// Halfword-wise unsigned minimum of two packed pairs.
__device__ __forceinline__ uint32_t min_u16x2(uint32_t a, uint32_t b) {
    uint32_t r;
    asm("min.u16x2 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(b));
    return r;
}

// hi32(a * b) + c, signed
__device__ __forceinline__ int mad_hi_s32(uint32_t a, int b, int c) {
    int d;
    asm("mad.hi.s32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(c));
    return d;
}

constexpr int kW2Warps = 8;
constexpr int kW2BlocksPerSM = 3;
constexpr int kW2LaneWords = 16;                      // words per lane and chunk
constexpr uint32_t kW2ChunkWords = 32u * kW2LaneWords;  // words per warp and chunk
// Table entry v of copy c at byte offset 256 v + 8 c, c = lane % 16: the shared
// address of byte k of a word w is one byte permute (byte k of w above the
// copy offset).  The 16 lanes of a half-warp (one 8-byte shared-memory
// transaction) read banks 2c, 2c + 1, whatever bytes they look up.
constexpr int kW2TableBytes = 256 * 256;

// Running sums of one lane over the words of its chunk: P = running step
// before the current word (relative to the lane's first bit); M2, Mz and SPw
// accumulate the square sums, the linear sums and the word-start prefixes
// (with constant offsets removed once per chunk); ext is the packed pair of
// extremes of the lane's running step, biased by kW2Bias.
struct W2Lane {
    int P;
    uint32_t M2, Mz;
    int SPw;
    uint32_t ext;
};

// One 32-site word w.  With a_j the running step inside the word (j = 0..31)
// and P the lane's running step before it, the word adds
//   sum (P + a_j) = 32 P + A1,  sum (P + a_j)^2 = P (32 P + 2 A1) + A2.
// Byte k (P_k = running step before it inside the word, P_0 = 0) contributes
// 8 P_k + t1 to A1 and 8 P_k^2 + 2 P_k t1 + t2 to A2.  u = 8 P_k + .x is
// 8 P_k + 2 t1 in its low 17 bits (the t2 and n fields only add multiples of
// 2^17), so
//   acc2 = 2^16 + sum_{k>=1} u P_k = 2^16 + V (mod 2^17), |V| <= 3 * 264 * 24 < 2^16,
// with V = sum (8 P_k^2 + 2 P_k t1), A2 = V + sum t2 and 2 A1 = 16 sum P_k + sum 2 t1.
// P_{k+1} = P_k + n is one multiply-high of .x.
__device__ __forceinline__ void w2_word(const unsigned char *tab, uint32_t slot, uint32_t w, W2Lane &a) {
    const uint2 e0 = *reinterpret_cast<const uint2 *>(tab + __byte_perm(w, slot, 0x6504));
    const uint2 e1 = *reinterpret_cast<const uint2 *>(tab + __byte_perm(w, slot, 0x6514));
    const uint2 e2 = *reinterpret_cast<const uint2 *>(tab + __byte_perm(w, slot, 0x6524));
    const uint2 e3 = *reinterpret_cast<const uint2 *>(tab + __byte_perm(w, slot, 0x6534));
    // extremes: .y + P_k (1 - 2^16) = (min + bias + P_k) | (bias - max - P_k) << 16
    const int p1 = mad_hi_s32(e0.x, 32, 0);
    uint32_t u = static_cast<uint32_t>(p1) * 8u + e1.x;
    uint32_t acc2 = u * static_cast<uint32_t>(p1) + 0x10000u;
    const uint32_t c1 = e1.y + static_cast<uint32_t>(p1) * 0xFFFF0001u;
    const int p2 = mad_hi_s32(e1.x, 32, p1);
    u = static_cast<uint32_t>(p2) * 8u + e2.x;
    acc2 += u * static_cast<uint32_t>(p2);
    const uint32_t c2 = e2.y + static_cast<uint32_t>(p2) * 0xFFFF0001u;
    const int p3 = mad_hi_s32(e2.x, 32, p2);
    u = static_cast<uint32_t>(p3) * 8u + e3.x;
    acc2 += u * static_cast<uint32_t>(p3);
    const uint32_t c3 = e3.y + static_cast<uint32_t>(p3) * 0xFFFF0001u;
    const int p4 = mad_hi_s32(e3.x, 32, p3);
    const uint32_t ext = min_u16x2(min_u16x2(e0.y, c1), min_u16x2(c2, c3));
    // S = sum .x + 512: Sl = sum 2 t1 + 512, bits 17..26 sum t2
    const uint32_t S = e0.x + e1.x + e2.x + e3.x + 512u;
    const uint32_t Sl = S & 0x1FFFFu, T2 = (S >> 17) & 0x3FFu;
    const uint32_t SP = static_cast<uint32_t>(p1 + p2 + p3);
    const uint32_t tw = SP * 16u + Sl;  // 2 A1 + 512
    // lane sums: zp = 32 P + 2 A1 + 512, P zp + Vb + t2 = (word's square sum)
    // + 512 P + 2^16; the offsets are removed at the end of the chunk
    const uint32_t P = static_cast<uint32_t>(a.P);
    const uint32_t zp = P * 32u + tw;
    a.M2 = zp * P + a.M2 + (acc2 & 0x1FFFFu) + T2;
    a.Mz += zp;
    a.SPw += a.P;
    a.ext = min_u16x2(a.ext, ext + P * 0xFFFF0001u);
    a.P += p4;
}

// The lane's kW2LaneWords words of the chunk at word w0 of a row (16-byte
// loads where the row allows them); words past the row's end read as 0 and
// are not counted.
__device__ __forceinline__ void load_lane(const uint32_t *row, uint32_t w, uint32_t wpr, bool vec_ok,
                                          uint32_t (&v)[kW2LaneWords]) {
    if (vec_ok && w + kW2LaneWords <= wpr) {
#pragma unroll
        for (int i = 0; i < kW2LaneWords / 4; ++i) {
            const uint4 q = *reinterpret_cast<const uint4 *>(row + w + 4 * i);
            v[4 * i] = q.x;
            v[4 * i + 1] = q.y;
            v[4 * i + 2] = q.z;
            v[4 * i + 3] = q.w;
        }
    } else {
#pragma unroll
        for (int i = 0; i < kW2LaneWords; ++i) v[i] = (w + i < wpr) ? row[w + i] : 0u;
    }
}

__global__ void __launch_bounds__(kW2Warps * 32, kW2BlocksPerSM)
    w2_rows_kernel(const uint32_t *lat, uint32_t L, uint32_t nrows, uint32_t plane_rows, W2RowSums *rows) {
    extern __shared__ __align__(16) unsigned char w2_table[];
    for (int i = threadIdx.x; i < 256; i += blockDim.x) {
        const uint2 e = byte_entry(static_cast<uint32_t>(i));
#pragma unroll
        for (int c = 0; c < 16; ++c) *reinterpret_cast<uint2 *>(w2_table + 256 * i + 8 * c) = e;
    }
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const uint32_t slot = 8u * static_cast<uint32_t>(lane & 15);
    const uint32_t wpr = L >> 5;
    const uint32_t *Yp = lat + static_cast<size_t>(plane_rows) * wpr;
    // 16-byte loads need every row to start on a 16-byte boundary
    const bool vec_ok = (wpr % 4u) == 0u && (reinterpret_cast<uintptr_t>(lat) % 16u) == 0u;
    // The warp's rows y0, y0 + stride, ... are taken chunk by chunk (chunks of
    // kW2ChunkWords words, lane i on words 16i..16i+15 of the chunk); the next
    // chunk's loads, across row ends too, are issued before the current chunk
    // is reduced.
    const uint32_t stride = gridDim.x * kW2Warps;
    const uint32_t nchunks = (wpr + kW2ChunkWords - 1) / kW2ChunkWords;
    uint32_t y = blockIdx.x * kW2Warps + (threadIdx.x >> 5), c = 0;
    uint32_t v[kW2LaneWords], vn[kW2LaneWords];
    if (y < nrows) load_lane(lat + static_cast<size_t>(y) * wpr, kW2LaneWords * lane, wpr, vec_ok, v);
    long long base = 0;  // q just before the current chunk
    long long q1 = 0, q2 = 0;
    int qmin = 1 << 30, qmax = -(1 << 30);
    while (y < nrows) {
        const uint32_t w0 = c * kW2ChunkWords;
        const uint32_t w = w0 + kW2LaneWords * lane;
        const bool last = c + 1 == nchunks;
        const uint32_t ny = last ? y + stride : y, nc = last ? 0u : c + 1;
        if (ny < nrows)
            load_lane(lat + static_cast<size_t>(ny) * wpr, nc * kW2ChunkWords + kW2LaneWords * lane, wpr, vec_ok, vn);
        W2Lane a{0, 0u, 0u, 0, 0xFFFFFFFFu};
        uint32_t nw = 0;
        if (w0 + kW2ChunkWords <= wpr) {
#pragma unroll
            for (int j = 0; j < kW2LaneWords; ++j) w2_word(w2_table, slot, v[j], a);
            nw = kW2LaneWords;
        } else {
#pragma unroll
            for (int j = 0; j < kW2LaneWords; ++j)
                if (w + j < wpr) {
                    w2_word(w2_table, slot, v[j], a);
                    ++nw;
                }
        }
        // lane-relative sums: sum q' and sum q'^2 over the lane's 32 nw sites
        // (|q'| <= 512, so both fit 32 bits), extremes and net step
        const int M2 = static_cast<int>(a.M2 - 512u * static_cast<uint32_t>(a.SPw) - 65536u * nw);
        const int M1 = static_cast<int>(a.Mz + 32u * static_cast<uint32_t>(a.SPw) - 512u * nw) / 2;
        const int step = a.P;
        int incl = step;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int n = __shfl_up_sync(kFull, incl, o);
            if (lane >= o) incl += n;
        }
        // lift to the row: q = B + q' with B = q before this lane's first bit
        const long long B = base + (incl - step);
        const long long nbits = 32ll * nw;
        q1 += nbits * B + M1;
        q2 += nbits * B * B + 2 * B * M1 + M2;
        if (nw > 0) {
            const int lmn = static_cast<int>(a.ext & 0xFFFFu) - static_cast<int>(kW2Bias);
            const int lmx = static_cast<int>(kW2Bias) - static_cast<int>(a.ext >> 16);
            qmin = min(qmin, static_cast<int>(B) + lmn);
            qmax = max(qmax, static_cast<int>(B) + lmx);
        }
        base += __shfl_sync(kFull, incl, 31);
        if (last) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                q1 += __shfl_xor_sync(kFull, q1, o);
                q2 += __shfl_xor_sync(kFull, q2, o);
            }
            qmin = __reduce_min_sync(kFull, qmin);
            qmax = __reduce_max_sync(kFull, qmax);
            if (lane == 0) {
                const uint32_t *row = lat + static_cast<size_t>(y) * wpr;
                const long long s0 = (row[0] & 1u) ? 1 : -1;
                const long long Ll = L;
                W2RowSums o;
                o.r1 = q1 - Ll * s0;
                o.r2 = q2 - 2 * s0 * q1 + Ll * s0 * s0;
                o.rmin = qmin - static_cast<int>(s0);
                o.rmax = qmax - static_cast<int>(s0);
                o.c = static_cast<int>(Yp[static_cast<size_t>(y) * wpr] & 1u);
                o.pad = 0;
                rows[y] = o;
            }
            base = 0;
            q1 = q2 = 0;
            qmin = 1 << 30;
            qmax = -(1 << 30);
        }
        y = ny;
        c = nc;
#pragma unroll
        for (int j = 0; j < kW2LaneWords; ++j) v[j] = vn[j];
    }
}

// Pass 2 runs in two kernels.  Pass 2a: one block per kW2BlockRows rows
// computes, relative to the height h0 of its first row, the sums
//   A = sum_y (L h0l + R1),  Q = sum_y (L h0l^2 + 2 h0l R1 + R2)
// (h0l = h0(y) - h0(first row)), the extremes of h0l + r and the rise of h0l
// to its last row, and stores them in place of its first row record.  Pass 2b
// (one block) scans the rises for each block's first-row height H and adds
// S1 = sum (A + L n H), S2 = sum (Q + 2 H A + L n H^2) over the blocks
// (n rows each) in 128-bit integers.
constexpr int kW2BlockRows = 256;
constexpr int kW2CombineThreads = 1024;

// The record of one pass-2a block, stored over its first row record.
struct W2BlockSums {
    long long a;                 // A
    unsigned long long q_lo;     // Q (>= 0: a sum of squared heights), bits 0..63
    unsigned int q_hi;           // bits 64..95 (Q < 2^70 for L <= 2^20)
    int lo, hi;                  // extremes of h0l + r over the block's rows
    int ec;                      // 2 h0l(last row) + Y(0, first row)
};
static_assert(sizeof(W2BlockSums) == sizeof(W2RowSums), "a block record replaces one row record");

// 128-bit unsigned sum of (lo, hi) pairs over a warp, in lane 0.
__device__ __forceinline__ void warp_sum_u128(unsigned long long &lo, unsigned long long &hi) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long l2 = __shfl_down_sync(kFull, lo, o);
        const unsigned long long h2 = __shfl_down_sync(kFull, hi, o);
        const unsigned long long nl = lo + l2;
        hi = hi + h2 + (nl < lo ? 1ull : 0ull);
        lo = nl;
    }
}

__global__ void __launch_bounds__(kW2BlockRows)
    w2_block_kernel(W2RowSums *rows, uint32_t L, uint32_t nrows) {
    __shared__ int wsum[kW2BlockRows / 32];
    __shared__ long long sa[kW2BlockRows / 32];
    __shared__ unsigned long long sqlo[kW2BlockRows / 32], sqhi[kW2BlockRows / 32];
    __shared__ int slo[kW2BlockRows / 32], shi[kW2BlockRows / 32];
    __shared__ int last_h0l;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t y0 = blockIdx.x * kW2BlockRows, y = y0 + tid;
    const uint32_t n = min(static_cast<uint32_t>(kW2BlockRows), nrows - y0);
    const bool valid = static_cast<uint32_t>(tid) < n;
    W2RowSums r{};
    if (valid) r = rows[y];
    // column step into row y from row y - 1 (none into the block's first row)
    int incl = (valid && tid > 0) ? (r.c ? 1 : -1) : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int v = __shfl_up_sync(kFull, incl, o);
        if (lane >= o) incl += v;
    }
    if (lane == 31) wsum[warp] = incl;
    __syncthreads();
    int before = 0;
    for (int w = 0; w < warp; ++w) before += wsum[w];
    const long long h = before + incl;  // h0l(y)
    if (static_cast<uint32_t>(tid) == n - 1) last_h0l = static_cast<int>(h);
    const long long Ll = L;
    long long a = 0;
    unsigned long long qlo = 0, qhi = 0;
    int lo = 1 << 30, hi = -(1 << 30);
    if (valid) {
        a = Ll * h + r.r1;
        // sum_x (h0l + r(x))^2 >= 0; |terms| < 2^63 for L <= 2^20
        const __int128 q = static_cast<__int128>(Ll * h * h) + static_cast<__int128>(2 * h * r.r1) +
                           static_cast<__int128>(r.r2);
        qlo = static_cast<unsigned long long>(q);
        qhi = static_cast<unsigned long long>(q >> 64);
        lo = static_cast<int>(h) + r.rmin;
        hi = static_cast<int>(h) + r.rmax;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) a += __shfl_down_sync(kFull, a, o);
    warp_sum_u128(qlo, qhi);
    lo = __reduce_min_sync(kFull, lo);
    hi = __reduce_max_sync(kFull, hi);
    if (lane == 0) {
        sa[warp] = a;
        sqlo[warp] = qlo;
        sqhi[warp] = qhi;
        slo[warp] = lo;
        shi[warp] = hi;
    }
    __syncthreads();
    if (tid == 0) {
        W2BlockSums b;
        b.a = 0;
        unsigned __int128 q = 0;
        b.lo = 1 << 30;
        b.hi = -(1 << 30);
        for (int w = 0; w < kW2BlockRows / 32; ++w) {
            b.a += sa[w];
            q += (static_cast<unsigned __int128>(sqhi[w]) << 64) | sqlo[w];
            b.lo = min(b.lo, slo[w]);
            b.hi = max(b.hi, shi[w]);
        }
        b.q_lo = static_cast<unsigned long long>(q);
        b.q_hi = static_cast<unsigned int>(q >> 64);
        b.ec = 2 * last_h0l + r.c;  // thread 0 holds the block's first row
        *reinterpret_cast<W2BlockSums *>(rows + y0) = b;
    }
}

__global__ void __launch_bounds__(kW2CombineThreads)
    w2_combine_kernel(const W2RowSums *rows, uint32_t L, uint32_t nrows, W2Result *out) {
    __shared__ long long part[kW2CombineThreads];
    __shared__ unsigned long long s2lo[kW2CombineThreads / 32], s2hi[kW2CombineThreads / 32];
    __shared__ long long s1w[kW2CombineThreads / 32], low[kW2CombineThreads / 32], hiw[kW2CombineThreads / 32];
    const int tid = threadIdx.x;
    const uint32_t nb = (nrows + kW2BlockRows - 1) / kW2BlockRows;
    const uint32_t per = (nb + kW2CombineThreads - 1) / kW2CombineThreads;
    const uint32_t b_begin = min(nb, tid * per), b_end = min(nb, (tid + 1) * per);
    auto rec = [&](uint32_t b) {
        return *reinterpret_cast<const W2BlockSums *>(rows + static_cast<size_t>(b) * kW2BlockRows);
    };
    // rise of h0 from the last row of block b - 1 to the last row of block b
    auto rise = [](const W2BlockSums &r, uint32_t b) {
        return static_cast<long long>(r.ec >> 1) + (b > 0 ? ((r.ec & 1) ? 1 : -1) : 0);
    };
    long long local = 0;
    for (uint32_t b = b_begin; b < b_end; ++b) local += rise(rec(b), b);
    part[tid] = local;
    __syncthreads();
    for (int o = 1; o < kW2CombineThreads; o <<= 1) {
        const long long v = (tid >= o) ? part[tid - o] : 0;
        __syncthreads();
        part[tid] += v;
        __syncthreads();
    }
    long long last = part[tid] - local;  // h0 of the last row before b_begin
    __int128 S1 = 0, S2 = 0;
    long long lo = 1ll << 62, hi = -(1ll << 62);
    const long long Ll = L;
    for (uint32_t b = b_begin; b < b_end; ++b) {
        const W2BlockSums r = rec(b);
        const long long H = last + (b > 0 ? ((r.ec & 1) ? 1 : -1) : 0);  // h0 of the block's first row
        const long long n = min(static_cast<uint32_t>(kW2BlockRows), nrows - b * kW2BlockRows);
        const __int128 Q = static_cast<__int128>((static_cast<unsigned __int128>(r.q_hi) << 64) | r.q_lo);
        S1 += static_cast<__int128>(r.a) + static_cast<__int128>(Ll * n) * H;
        S2 += Q + static_cast<__int128>(2 * H) * r.a + static_cast<__int128>(Ll * n) * H * H;
        lo = min(lo, H + r.lo);
        hi = max(hi, H + r.hi);
        last = H + (r.ec >> 1);
    }
    if (b_end == nb && b_begin < b_end) out->e_last = last;  // h0 of the last row
    // block reduction of S1 (fits 64 bits for L <= 2^20), S2 (128 bits), extremes
    long long s1 = static_cast<long long>(S1);
    unsigned long long s2l = static_cast<unsigned long long>(S2);
    unsigned long long s2h = static_cast<unsigned long long>(S2 >> 64);
    for (int o = 16; o > 0; o >>= 1) {
        s1 += __shfl_down_sync(kFull, s1, o);
        lo = min(lo, __shfl_down_sync(kFull, lo, o));
        hi = max(hi, __shfl_down_sync(kFull, hi, o));
    }
    warp_sum_u128(s2l, s2h);
    if ((tid & 31) == 0) {
        s1w[tid >> 5] = s1;
        s2lo[tid >> 5] = s2l;
        s2hi[tid >> 5] = s2h;
        low[tid >> 5] = lo;
        hiw[tid >> 5] = hi;
    }
    __syncthreads();
    if (tid == 0) {
        long long a1 = 0, amn = 1ll << 62, amx = -(1ll << 62);
        unsigned __int128 a2 = 0;
        for (int w = 0; w < kW2CombineThreads / 32; ++w) {
            a1 += s1w[w];
            a2 += (static_cast<unsigned __int128>(s2hi[w]) << 64) | s2lo[w];
            amn = min(amn, low[w]);
            amx = max(amx, hiw[w]);
        }
        out->s1 = a1;
        out->s2_lo = static_cast<unsigned long long>(a2);
        out->s2_hi = static_cast<unsigned long long>(a2 >> 64);
        out->lo = amn;
        out->hi = amx;
        out->hmax = max(amn < 0 ? -amn : amn, amx < 0 ? -amx : amx);
        out->f0 = (rec(0).ec & 1) ? 1 : -1;
    }
}

// Interleave two 4-bit values: a0 b0 a1 b1 a2 b2 a3 b3 (LSB first).
__device__ __forceinline__ uint32_t interleave4(uint32_t a, uint32_t b) {
    uint32_t r = 0;
#pragma unroll
    for (int i = 0; i < 4; ++i) r |= (((a >> i) & 1u) << (2 * i)) | (((b >> i) & 1u) << (2 * i + 1));
    return r;
}

__global__ void pack_canonical_kernel(const uint32_t *lat, uint32_t L, uint32_t cy0, uint32_t ncy,
                                      uint32_t *out) {
    const uint32_t wpr = L >> 5, cpr = L >> 2;  // canonical words per canonical row
    const uint32_t *Yp = lat + static_cast<size_t>(L) * wpr;
    const uint64_t n = static_cast<uint64_t>(ncy) * cpr;
    for (uint64_t i = blockIdx.x * static_cast<uint64_t>(blockDim.x) + threadIdx.x; i < n;
         i += static_cast<uint64_t>(gridDim.x) * blockDim.x) {
        const uint32_t cy = cy0 + static_cast<uint32_t>(i / cpr), cx = static_cast<uint32_t>(i % cpr);
        const uint32_t w = (4u * cx) >> 5, b = (4u * cx) & 31u;
        uint32_t v = 0;
#pragma unroll
        for (int yy = 0; yy < 4; ++yy) {
            const size_t ro = static_cast<size_t>(4u * cy + yy) * wpr + w;
            v |= interleave4((lat[ro] >> b) & 0xFu, (Yp[ro] >> b) & 0xFu) << (8 * yy);
        }
        out[i] = v;
    }
}

__global__ void unpack_canonical_kernel(const uint32_t *in, uint32_t L, uint32_t cy0, uint32_t ncy,
                                        uint32_t *lat) {
    // one thread per planar word pair (X and Y) of lattice rows 4*cy0 .. 4*(cy0+ncy)-1
    const uint32_t wpr = L >> 5, cpr = L >> 2;
    uint32_t *Yp = lat + static_cast<size_t>(L) * wpr;
    const uint64_t n = static_cast<uint64_t>(ncy) * 4u * wpr;
    for (uint64_t i = blockIdx.x * static_cast<uint64_t>(blockDim.x) + threadIdx.x; i < n;
         i += static_cast<uint64_t>(gridDim.x) * blockDim.x) {
        const uint32_t lr = static_cast<uint32_t>(i / wpr), w = static_cast<uint32_t>(i % wpr);
        const uint32_t y = 4u * cy0 + lr, yy = y & 3u;
        uint32_t xv = 0, yv = 0;
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            const uint32_t word = in[static_cast<size_t>(lr >> 2) * cpr + 8u * w + c] >> (8u * yy);
#pragma unroll
            for (int xx = 0; xx < 4; ++xx) {
                xv |= ((word >> (2 * xx)) & 1u) << (4 * c + xx);
                yv |= ((word >> (2 * xx + 1)) & 1u) << (4 * c + xx);
            }
        }
        lat[static_cast<size_t>(y) * wpr + w] = xv;
        Yp[static_cast<size_t>(y) * wpr + w] = yv;
    }
}

// One thread per counter slot (kNetSlots threads), then a block reduction.
__global__ void __launch_bounds__(kNetSlots)
    net_sum_kernel(const unsigned long long *net, const unsigned long long *draws, const unsigned long long *tails,
                   long long *out) {
    __shared__ long long part[3][kNetSlots / 32];
    const int i = threadIdx.x;
    long long s = static_cast<long long>(net[i]), d = static_cast<long long>(draws[i]),
              b = static_cast<long long>(tails[i]);
    for (int o = 16; o > 0; o >>= 1) {
        s += __shfl_down_sync(kFull, s, o);
        d += __shfl_down_sync(kFull, d, o);
        b += __shfl_down_sync(kFull, b, o);
    }
    if ((i & 31) == 0) {
        part[0][i >> 5] = s;
        part[1][i >> 5] = d;
        part[2][i >> 5] = b;
    }
    __syncthreads();
    if (i < 3) {
        long long t = 0;
        for (int w = 0; w < kNetSlots / 32; ++w) t += part[i][w];
        out[i] = t;
    }
}

int grid_for(uint64_t n, int threads) {
    const uint64_t b = (n + threads - 1) / threads;
    return static_cast<int>(b < 152ull * 32 ? (b ? b : 1) : 152ull * 32);
}

}  // namespace

cudaError_t launch_init_flat(uint32_t *lat, uint32_t L, cudaStream_t st) {
    return launch_init_flat_rows(lat, L, L, st);
}

cudaError_t launch_init_flat_rows(uint32_t *lat, uint32_t L, uint32_t rows, cudaStream_t st) {
    const uint32_t wpr = L >> 5;
    const uint64_t n = 2ull * rows * wpr;
    init_flat_kernel<<<grid_for(n, 256), 256, 0, st>>>(lat, rows, n, wpr);
    return cudaGetLastError();
}

cudaError_t launch_w2(const uint32_t *lat, uint32_t L, W2RowSums *rows, W2Result *out,
                      cudaStream_t st) {
    return launch_w2_rows(lat, L, L, L, rows, out, st);
}

cudaError_t launch_w2_rows(const uint32_t *lat, uint32_t L, uint32_t nrows, uint32_t plane_rows, W2RowSums *rows,
                           W2Result *out, cudaStream_t st) {
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
        e = cudaFuncSetAttribute(w2_rows_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kW2TableBytes);
        if (e != cudaSuccess) return e;
        smem_set[dev] = true;
    }
    const uint64_t want = (static_cast<uint64_t>(nrows) + kW2Warps - 1) / kW2Warps;
    const uint64_t wave = static_cast<uint64_t>(sms[dev]) * kW2BlocksPerSM;
    const int blocks = static_cast<int>(want < wave ? want : wave);
    w2_rows_kernel<<<blocks, kW2Warps * 32, kW2TableBytes, st>>>(lat, L, nrows, plane_rows, rows);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    w2_block_kernel<<<(nrows + kW2BlockRows - 1) / kW2BlockRows, kW2BlockRows, 0, st>>>(rows, L, nrows);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    w2_combine_kernel<<<1, kW2CombineThreads, 0, st>>>(rows, L, nrows, out);
    return cudaGetLastError();
}

cudaError_t launch_pack_canonical(const uint32_t *lat, uint32_t L, uint32_t cy0, uint32_t ncy,
                                  uint32_t *out, cudaStream_t st) {
    pack_canonical_kernel<<<grid_for(static_cast<uint64_t>(ncy) * (L >> 2), 256), 256, 0, st>>>(
        lat, L, cy0, ncy, out);
    return cudaGetLastError();
}

cudaError_t launch_unpack_canonical(const uint32_t *in, uint32_t L, uint32_t cy0, uint32_t ncy,
                                    uint32_t *lat, cudaStream_t st) {
    unpack_canonical_kernel<<<grid_for(static_cast<uint64_t>(ncy) * 4u * (L >> 5), 256), 256, 0,
                              st>>>(in, L, cy0, ncy, lat);
    return cudaGetLastError();
}

cudaError_t launch_net_sum(const unsigned long long *net, const unsigned long long *draws,
                           const unsigned long long *tails, long long *out, cudaStream_t st) {
    net_sum_kernel<<<1, kNetSlots, 0, st>>>(net, draws, tails, out);
    return cudaGetLastError();
}

}  // namespace oct
