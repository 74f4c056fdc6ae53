// Lattice-wide kernels: flat start, exact roughness, layout conversion.
//
// Roughness (Eq. (3), mean over the L^2 sites): heights relative to h(0,0)=0,
//   h(0,y) = sum_{y'=1..y} (2 Y(0,y') - 1),
//   h(x,y) = h(0,y) + r(x,y),  r(x,y) = sum_{x'=1..x} (2 X(x',y) - 1).
// Pass 1 (one warp per row): with q(x) = sum_{x'=0..x} (2X(x',y)-1) and
// s0 = 2X(0,y)-1, r = q - s0, so the row sums of r and r^2 follow from those
// of q, which a warp computes with 128-bit coalesced loads, a warp scan of
// per-lane step counts and a 256-entry byte table (sum of the running step
// inside a byte, its square, its extremes).  Pass 2 (one block): a scan of the
// column bits gives h(0,y), and S1 = sum_y (L h0 + R1), S2 = sum_y (L h0^2 +
// 2 h0 R1 + R2) accumulate in 128-bit integers.  Per-row terms are bounded by
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

// Byte table: for byte value v, with running step e_i = sum_{j<=i} (2 b_j - 1),
// i = 0..7:
//   .x = sum e_i (signed byte) | net e_7 << 8 (signed byte) | sum e_i^2 << 16
//   .y = the extremes as two biased 16-bit halves for one packed minimum:
//        (min e_i + kW2Bias) | (kW2Bias - max e_i) << 16
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
    r.x = (static_cast<uint32_t>(s1) & 0xFFu) | ((static_cast<uint32_t>(e) & 0xFFu) << 8) |
          (static_cast<uint32_t>(s2) << 16);
    r.y = (kW2Bias + static_cast<uint32_t>(mn)) | ((kW2Bias - static_cast<uint32_t>(mx)) << 16);
    return r;
}

__device__ __forceinline__ int sbyte(uint32_t x, int k) {
    return static_cast<int>(static_cast<signed char>(static_cast<unsigned char>(x >> (8 * k))));
}

// Halfword-wise unsigned minimum of two packed pairs.
__device__ __forceinline__ uint32_t min_u16x2(uint32_t a, uint32_t b) {
    uint32_t r;
    asm("min.u16x2 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(b));
    return r;
}

constexpr int kW2Warps = 8;

// The 4 words w..w+3 of a row (one 16-byte load where the row allows it);
// words past the row's end read as 0 and are not counted.
__device__ __forceinline__ uint4 load_chunk(const uint32_t *row, uint32_t w, uint32_t wpr, bool vec_ok) {
    uint4 v = make_uint4(0u, 0u, 0u, 0u);
    if (vec_ok && w + 3u < wpr) {
        v = *reinterpret_cast<const uint4 *>(row + w);
    } else if (w < wpr) {
        v.x = row[w];
        if (w + 1u < wpr) v.y = row[w + 1];
        if (w + 2u < wpr) v.z = row[w + 2];
        if (w + 3u < wpr) v.w = row[w + 3];
    }
    return v;
}

// Copies of the byte table: lane l reads copy l % 16, entry e of copy c at
// uint2 index 16 e + c, i.e. banks 2c and 2c + 1.  The 16 lanes of a
// half-warp (one 8-byte shared-memory transaction) then never share a bank,
// whatever bytes they look up.
constexpr int kW2TableCopies = 16;

__global__ void __launch_bounds__(kW2Warps * 32)
    w2_rows_kernel(const uint32_t *lat, uint32_t L, uint32_t nrows, uint32_t plane_rows, W2RowSums *rows) {
    __shared__ uint2 table[256 * kW2TableCopies];
    for (int i = threadIdx.x; i < 256; i += blockDim.x) {
        const uint2 e = byte_entry(static_cast<uint32_t>(i));
#pragma unroll
        for (int c = 0; c < kW2TableCopies; ++c) table[i * kW2TableCopies + c] = e;
    }
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const uint2 *const my_table = table + (lane % kW2TableCopies);
    const uint32_t wpr = L >> 5;
    const uint32_t *Yp = lat + static_cast<size_t>(plane_rows) * wpr;
    // 16-byte loads need every row to start on a 16-byte boundary
    const bool vec_ok = (wpr % 4u) == 0u && (reinterpret_cast<uintptr_t>(lat) % 16u) == 0u;
    for (uint32_t y = blockIdx.x * kW2Warps + (threadIdx.x >> 5); y < nrows; y += gridDim.x * kW2Warps) {
        const uint32_t *row = lat + static_cast<size_t>(y) * wpr;
        long long base = 0;  // q just before the current chunk
        long long q1 = 0, q2 = 0;
        int qmin = 1 << 30, qmax = -(1 << 30);
        // Chunks of 128 words: lane i takes words 4i..4i+3; the next chunk's
        // load is issued before the current one is reduced.
        uint4 v = load_chunk(row, 4u * lane, wpr, vec_ok);
        for (uint32_t w0 = 0; w0 < wpr; w0 += 128u) {
            const uint32_t w = w0 + 4u * lane;
            const uint4 vn = load_chunk(row, w + 128u, wpr, vec_ok);
            const int nw = (w < wpr) ? static_cast<int>(min(4u, wpr - w)) : 0;
            const int nbits = 32 * nw;
            const int step = 2 * (__popc(v.x) + __popc(v.y) + __popc(v.z) + __popc(v.w)) - nbits;
            int incl = step;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int n = __shfl_up_sync(kFull, incl, o);
                if (lane >= o) incl += n;
            }
            // Lane-local running sum a (0 at the lane's first bit) in 32 bits:
            // |a| <= 128, sum a <= 2^14, sum a^2 <= 2^21.
            // ext: running packed minimum of (a + min e + bias | bias - a - max e),
            // both halves within [bias - 136, bias + 136]
            int a = 0, l1 = 0, l2 = 0;
            uint32_t ext = 0xFFFFFFFFu;
            const uint32_t words[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                if (j >= nw) break;
#pragma unroll
                for (int byte = 0; byte < 4; ++byte) {
                    const uint2 te = my_table[((words[j] >> (8 * byte)) & 0xFFu) * kW2TableCopies];
                    const int t1 = sbyte(te.x, 0), net = sbyte(te.x, 1);
                    l1 += 8 * a + t1;
                    l2 += a * (8 * a + 2 * t1) + static_cast<int>(te.x >> 16);
                    // + a in the low half, - a in the high half (a * (1 - 2^16))
                    ext = min_u16x2(ext, te.y + static_cast<uint32_t>(a) * 0xFFFF0001u);
                    a += net;
                }
            }
            // lift to the row: q = B + a with B = q before this lane's first bit
            const long long B = base + (incl - step);
            q1 += static_cast<long long>(nbits) * B + l1;
            q2 += static_cast<long long>(nbits) * B * B + 2 * B * l1 + l2;
            if (nw > 0) {
                const int lmn = static_cast<int>(ext & 0xFFFFu) - static_cast<int>(kW2Bias);
                const int lmx = static_cast<int>(kW2Bias) - static_cast<int>(ext >> 16);
                qmin = min(qmin, static_cast<int>(B) + lmn);
                qmax = max(qmax, static_cast<int>(B) + lmx);
            }
            base += __shfl_sync(kFull, incl, 31);
            v = vn;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            q1 += __shfl_xor_sync(kFull, q1, o);
            q2 += __shfl_xor_sync(kFull, q2, o);
        }
        qmin = __reduce_min_sync(kFull, qmin);
        qmax = __reduce_max_sync(kFull, qmax);
        if (lane == 0) {
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
    }
}

constexpr int kFinalThreads = 1024;

// Pass 2 over nrows row records of rows of length L: heights h0 = sum of the
// column steps of rows 1..y (row 0 at 0), S1, S2 (128-bit), the extremes of
// h0 + r, h0 of the last row and the first row's column step.
__global__ void __launch_bounds__(kFinalThreads)
    w2_final_kernel(const W2RowSums *rows, uint32_t L, uint32_t nrows, W2Result *out) {
    __shared__ long long part[kFinalThreads];
    __shared__ unsigned long long s2lo[kFinalThreads / 32], s2hi[kFinalThreads / 32];
    __shared__ long long s1w[kFinalThreads / 32], low[kFinalThreads / 32], hiw[kFinalThreads / 32];
    const int tid = threadIdx.x;
    const uint32_t per = (nrows + kFinalThreads - 1) / kFinalThreads;
    const uint32_t y_begin = min(nrows, tid * per), y_end = min(nrows, (tid + 1) * per);
    // column steps 2c-1 for rows 1..y (row 0 contributes nothing)
    long long local = 0;
    for (uint32_t y = y_begin; y < y_end; ++y)
        if (y > 0) local += rows[y].c ? 1 : -1;
    part[tid] = local;
    __syncthreads();
    // exclusive scan of the per-thread column sums (Hillis-Steele on shared memory)
    for (int o = 1; o < kFinalThreads; o <<= 1) {
        const long long v = (tid >= o) ? part[tid - o] : 0;
        __syncthreads();
        part[tid] += v;
        __syncthreads();
    }
    long long h0 = part[tid] - local;
    if (tid == kFinalThreads - 1) out->e_last = part[tid];  // h0 of the last row
    __int128 S1 = 0, S2 = 0;
    long long lo = 1ll << 62, hi = -(1ll << 62);
    const long long Ll = L;
    for (uint32_t y = y_begin; y < y_end; ++y) {
        const W2RowSums r = rows[y];
        if (y > 0) h0 += r.c ? 1 : -1;
        S1 += static_cast<__int128>(Ll * h0 + r.r1);
        S2 += static_cast<__int128>(Ll * h0 * h0) + static_cast<__int128>(2 * h0 * r.r1) +
              static_cast<__int128>(r.r2);
        lo = min(lo, h0 + r.rmin);
        hi = max(hi, h0 + r.rmax);
    }
    // block reduction of S1 (fits 64 bits for L <= 2^20), S2 (128 bits), extremes
    long long s1 = static_cast<long long>(S1);
    unsigned long long s2l = static_cast<unsigned long long>(S2);
    unsigned long long s2h = static_cast<unsigned long long>(S2 >> 64);
    for (int o = 16; o > 0; o >>= 1) {
        s1 += __shfl_down_sync(kFull, s1, o);
        const unsigned long long lo2 = __shfl_down_sync(kFull, s2l, o);
        const unsigned long long hi2 = __shfl_down_sync(kFull, s2h, o);
        const unsigned long long nlo = s2l + lo2;
        s2h = s2h + hi2 + (nlo < s2l ? 1ull : 0ull);
        s2l = nlo;
        lo = min(lo, __shfl_down_sync(kFull, lo, o));
        hi = max(hi, __shfl_down_sync(kFull, hi, o));
    }
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
        for (int w = 0; w < kFinalThreads / 32; ++w) {
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
        out->f0 = rows[0].c ? 1 : -1;
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

__global__ void net_sum_kernel(const unsigned long long *net, const unsigned long long *draws,
                               const unsigned long long *tails, long long *out) {
    long long s = 0, d = 0, b = 0;
    for (int i = threadIdx.x; i < kNetSlots; i += 32) {
        s += static_cast<long long>(net[i]);
        d += static_cast<long long>(draws[i]);
        b += static_cast<long long>(tails[i]);
    }
    for (int o = 16; o > 0; o >>= 1) {
        s += __shfl_down_sync(kFull, s, o);
        d += __shfl_down_sync(kFull, d, o);
        b += __shfl_down_sync(kFull, b, o);
    }
    if (threadIdx.x == 0) {
        out[0] = s;
        out[1] = d;
        out[2] = b;
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
    // one wave of resident blocks (32 KB of table each), rows taken grid-stride
    static int sms = 0;
    if (sms == 0) {
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0)
            sms = 152;
    }
    const uint64_t want = (static_cast<uint64_t>(nrows) + kW2Warps - 1) / kW2Warps;
    const uint64_t wave = static_cast<uint64_t>(sms) * 6u;
    const int blocks = static_cast<int>(want < wave ? want : wave);
    w2_rows_kernel<<<blocks, kW2Warps * 32, 0, st>>>(lat, L, nrows, plane_rows, rows);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    w2_final_kernel<<<1, kFinalThreads, 0, st>>>(rows, L, nrows, out);
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
    net_sum_kernel<<<1, 32, 0, st>>>(net, draws, tails, out);
    return cudaGetLastError();
}

}  // namespace oct
