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
// Each lane takes 128 sites of the row (one 16-byte load per plane and
// lattice); a packed warp scan of both lattices' step counts gives the lane's
// starting q.  Inside the lane the running sums restart at 0 and are built one
// nibble pair at a time from two tables: for a nibble n, the sum of its four
// running steps and its net step; for a pair of nibbles, the sum of the
// products of their running steps.  The lane's local sums are lifted to the
// row's with one 64-bit multiply-add per lattice.
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

__global__ void __launch_bounds__(kAcWarps * 32)
    ac_rows_kernel(const uint32_t *lt, const uint32_t *ls, uint32_t L, AcRowSums *rows) {
    // sum_i a_i(n_t) a_i(n_s) for the nibble pair e = n_t | n_s << 4, one copy
    // per lane (entry e of lane l at word 32 e + l: every lane reads its own
    // bank, so the random lookups never conflict)
    __shared__ int pair_tab[256 * 32];
    __shared__ int2 nib_tab[16];   // (sum_i a_i(n), a_3(n)); 16 entries fill 32 banks once
    for (int i = threadIdx.x; i < 256 * 32; i += blockDim.x) {
        const uint32_t e = static_cast<uint32_t>(i) >> 5;
        int a[4], b[4];
        nibble_steps(e & 15u, a);
        nibble_steps(e >> 4, b);
        pair_tab[i] = a[0] * b[0] + a[1] * b[1] + a[2] * b[2] + a[3] * b[3];
        if (i < 16) {
            nibble_steps(static_cast<uint32_t>(i), a);
            nib_tab[i] = make_int2(a[0] + a[1] + a[2] + a[3], a[3]);
        }
    }
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int *const my_pairs = pair_tab + lane;
    const uint32_t wpr = L >> 5;
    const size_t plane = static_cast<size_t>(L) * wpr;
    const bool vec_ok = (wpr % 4u) == 0u && (reinterpret_cast<uintptr_t>(lt) % 16u) == 0u &&
                        (reinterpret_cast<uintptr_t>(ls) % 16u) == 0u;
    for (uint32_t y = blockIdx.x * kAcWarps + (threadIdx.x >> 5); y < L; y += gridDim.x * kAcWarps) {
        const size_t ro = static_cast<size_t>(y) * wpr;
        long long base_t = 0, base_s = 0;  // q just before the current chunk
        long long qt = 0, qs = 0, qts = 0;
        int nx = 0, ny = 0, mt = 0, ms = 0;
        for (uint32_t w0 = 0; w0 < wpr; w0 += 128u) {
            const uint32_t w = w0 + 4u * lane;
            uint32_t wt[4] = {0u, 0u, 0u, 0u}, ws[4] = {0u, 0u, 0u, 0u};
            uint32_t vt[4] = {0u, 0u, 0u, 0u}, vs[4] = {0u, 0u, 0u, 0u};
            int nbits = 0;
            if (vec_ok && w + 3u < wpr) {
                const uint4 a = *reinterpret_cast<const uint4 *>(lt + ro + w);
                const uint4 b = *reinterpret_cast<const uint4 *>(ls + ro + w);
                const uint4 c = *reinterpret_cast<const uint4 *>(lt + plane + ro + w);
                const uint4 d = *reinterpret_cast<const uint4 *>(ls + plane + ro + w);
                wt[0] = a.x; wt[1] = a.y; wt[2] = a.z; wt[3] = a.w;
                ws[0] = b.x; ws[1] = b.y; ws[2] = b.z; ws[3] = b.w;
                vt[0] = c.x; vt[1] = c.y; vt[2] = c.z; vt[3] = c.w;
                vs[0] = d.x; vs[1] = d.y; vs[2] = d.z; vs[3] = d.w;
                nbits = 128;
            } else {
#pragma unroll
                for (uint32_t j = 0; j < 4u; ++j)
                    if (w + j < wpr) {
                        wt[j] = lt[ro + w + j];
                        ws[j] = ls[ro + w + j];
                        vt[j] = lt[plane + ro + w + j];
                        vs[j] = ls[plane + ro + w + j];
                        nbits += 32;
                    }
            }
            // X words wt (lattice t), ws (lattice s); Y words vt, vs
            int pt = 0, ps = 0;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                pt += __popc(wt[j]);
                ps += __popc(ws[j]);
                nx += __popc(wt[j] & ws[j]);
                ny += __popc(vt[j] & vs[j]);
                mt += __popc(vt[j]);
                ms += __popc(vs[j]);
            }
            mt += pt;
            ms += ps;
            // Step counts of both lattices in one scan: |prefix| <= 4096, so the
            // t count fits the low 16 bits of a two's-complement packed word.
            const int st = 2 * pt - nbits, ss = 2 * ps - nbits;
            int incl = st + ss * 65536;
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
            const long long Bt = base_t + (incl_t - st), Bs = base_s + (incl_s - ss);
            // lane-local running sums (start at 0): sum a_t, sum a_s, sum a_t a_s
            int bt = 0, bs = 0, lst = 0, lss = 0, lc = 0;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                if (32 * j >= nbits) break;
#pragma unroll
                for (int k = 0; k < 8; ++k) {
                    const uint32_t nt = (wt[j] >> (4 * k)) & 15u, ns = (ws[j] >> (4 * k)) & 15u;
                    const int2 et = nib_tab[nt], es = nib_tab[ns];
                    lc += bt * (4 * bs + es.x) + bs * et.x + my_pairs[(nt | (ns << 4)) << 5];
                    lst += 4 * bt + et.x;
                    lss += 4 * bs + es.x;
                    bt += et.y;
                    bs += es.y;
                }
            }
            qts += static_cast<long long>(nbits) * Bt * Bs + Bt * lss + Bs * lst + lc;
            qt += static_cast<long long>(nbits) * Bt + lst;
            qs += static_cast<long long>(nbits) * Bs + lss;
            base_t += tot_t;
            base_s += tot_s;
        }
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
    const uint64_t want = (static_cast<uint64_t>(L) + kAcWarps - 1) / kAcWarps;
    const int blocks = static_cast<int>(want < 152ull * 8 ? want : 152ull * 8);
    ac_rows_kernel<<<blocks, kAcWarps * 32, 0, st>>>(lat_t, lat_s, L, rows);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    ac_block_kernel<<<(L + kAcBlockRows - 1) / kAcBlockRows, kAcBlockRows, 0, st>>>(rows, L);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    ac_combine_kernel<<<1, kAcCombineThreads, 0, st>>>(rows, L, out);
    return cudaGetLastError();
}

}  // namespace oct
