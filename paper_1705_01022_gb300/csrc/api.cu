// C ABI of the simulator (include/oct.h): argument checks, memory ownership,
// stream handling and the per-MCS launch sequence.  All arithmetic of the
// method runs in the kernels of dtrdt.cu and lattice.cu.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "../../include/oct.h"
#include "oct_internal.h"
#include "philox.cuh"

namespace {

thread_local std::string g_last_error;

int fail(int code, const std::string &msg) {
    g_last_error = msg;
    return code;
}

int cuda_fail(cudaError_t e, const char *what) {
    return fail(OCT_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define OCT_CUDA(call)                                   \
    do {                                                 \
        cudaError_t e_ = (call);                         \
        if (e_ != cudaSuccess) return cuda_fail(e_, #call); \
    } while (0)

// Acceptance threshold P32 = floor(p * 2^32) for 0 < p < 1 (the attempt is
// accepted iff its uniform 32-bit word is below it).
uint32_t threshold32(double p) { return static_cast<uint32_t>(std::floor(std::ldexp(p, 32))); }

constexpr int kEventPairs = 256;

}  // namespace

void oct::set_last_error(const std::string &msg) { g_last_error = msg; }

// C_h and C_s from the exact sums (numerators in 128-bit integers).
void oct::fill_ac(int64_t L, const oct::AcResult &r, oct_ac *out) {
    const __int128 N = static_cast<__int128>(L) * L;
    const __int128 cross =
        static_cast<__int128>((static_cast<unsigned __int128>(r.cross_hi) << 64) | r.cross_lo);
    const __int128 num_h = N * cross - static_cast<__int128>(r.sum_ht) * r.sum_hs;
    const __int128 M = 2 * N;
    const __int128 num_s = M * static_cast<__int128>(r.occ_x + r.occ_y) - static_cast<__int128>(r.m_t) * r.m_s;
    *out = oct_ac{};
    out->n_sites = static_cast<int64_t>(N);
    out->sum_ht = r.sum_ht;
    out->sum_hs = r.sum_hs;
    out->cross_lo = r.cross_lo;
    out->cross_hi = static_cast<int64_t>(r.cross_hi);
    out->occ_x = r.occ_x;
    out->occ_y = r.occ_y;
    out->m_t = r.m_t;
    out->m_s = r.m_s;
    out->c_h = static_cast<double>(num_h) / (static_cast<double>(N) * static_cast<double>(N));
    out->c_s = static_cast<double>(num_s) / (static_cast<double>(M) * static_cast<double>(M));
}

struct oct_sim {
    int64_t L = 0;
    double p = 0, q = 0;
    uint64_t seed = 0;
    int Bx = 0, By = 0, cx = 4, cy = 4;
    int scheme = 0;
    int64_t strip_row0 = 0, strip_rows = 0, held_rows = 0;  // strip_rows = 0: the whole lattice
    int next_k = 0;  // next device step of oct_device_step
    uint32_t *lat = nullptr;
    bool own_lat = false;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int device = 0;
    uint32_t *d_t = nullptr;
    unsigned long long *d_net = nullptr;    // kNetSlots flip, then draw, then tail-block counters
    long long *d_net_sum = nullptr;         // [net flips, acceptance draws, tail blocks]
    oct::W2RowSums *d_rows = nullptr;
    oct::W2Result *d_w2 = nullptr;
    void *h_small = nullptr;  // pinned: W2Result at 0, its net sum at 128, oct_get_stats' net sum at 192
    uint64_t t = 0;
    bool w2_pending = false;  // oct_measure_w2_async enqueued, oct_w2_wait not yet called
    uint64_t w2_t = 0;        // time of the pending measurement
    oct::StepArgs args{};
    bool any_random = false;
    // timing
    bool timing = false;
    std::vector<cudaEvent_t> ev;  // kEventPairs start/stop pairs
    int ev_used = 0;
    double step_ms = 0.0;
    int64_t step_launches = 0;
    int64_t draws = 0;  // acceptance draws counted up to the last measurement
    // two-time autocorrelations
    uint32_t *snap = nullptr;  // planar lattice at the waiting time
    int64_t snap_t = -1;
    oct::AcRowSums *d_ac_rows = nullptr;
    oct::AcResult *d_ac = nullptr;
};

namespace {

int flush_timing(oct_sim *s) {
    if (s->ev_used == 0) return OCT_OK;
    OCT_CUDA(cudaEventSynchronize(s->ev[2 * (s->ev_used - 1) + 1]));
    for (int i = 0; i < s->ev_used; ++i) {
        float ms = 0.f;
        OCT_CUDA(cudaEventElapsedTime(&ms, s->ev[2 * i], s->ev[2 * i + 1]));
        s->step_ms += ms;
    }
    s->ev_used = 0;
    return OCT_OK;
}

int validate(const oct_params *prm, int *Bx, int *By, int *cx, int *cy) {
    const int64_t L = prm->L;
    if (L < 64 || L > (int64_t{1} << 20) || (L % 64) != 0)
        return fail(OCT_EINVAL, "L must be a multiple of 64 in [64, 2^20]");
    if (!(prm->p >= 0.0 && prm->p <= 1.0) || !(prm->q >= 0.0 && prm->q <= 1.0))
        return fail(OCT_EINVAL, "p and q must lie in [0, 1]");
    *cx = prm->cx ? prm->cx : 4;
    *cy = prm->cy ? prm->cy : 4;
    const bool coarse = *cx != 4 || *cy != 4;
    if (coarse && !oct::cells_shape_supported(*cx, *cy))
        return fail(OCT_EUNSUPPORTED,
                    "thread cells: cx in {4, 8, 16, 32} and cy in {4, 8, 16} sites (4 x 16 included)");
    if (coarse && prm->scheme != OCT_SCHEME_DT)
        return fail(OCT_EUNSUPPORTED, "thread cells other than 4 x 4 sites are implemented for DTrDT only");
    if (prm->Bx || prm->By) {
        *Bx = prm->Bx;
        *By = prm->By;
    } else if (L % 128 == 0) {
        *Bx = 64;
        *By = 64;
    } else {
        *Bx = 32;
        *By = 16;
    }
    if (*Bx < 32 || *By < 16 || *Bx % 32 || *By % 16)
        return fail(OCT_EINVAL, "Bx must be a multiple of 32 and By a multiple of 16");
    if ((*Bx / 32) * (*By / 16) > 32)
        return fail(OCT_EINVAL, "a sub-tile may hold at most 32 groups of 32x16 sites");
    if (L % (2 * *Bx) || L % (2 * *By)) return fail(OCT_EINVAL, "L must be a multiple of 2Bx and 2By");
    if (prm->scheme != OCT_SCHEME_DT && prm->scheme != OCT_SCHEME_DB && prm->scheme != OCT_SCHEME_DTR)
        return fail(OCT_EINVAL, "scheme must be OCT_SCHEME_DT, OCT_SCHEME_DB or OCT_SCHEME_DTR");
    if (prm->strip_rows || prm->strip_row0 || prm->held_rows) {
        const int64_t t2 = 2 * static_cast<int64_t>(*By);
        if (prm->strip_rows <= 0 || prm->strip_rows % t2 || prm->strip_row0 < 0 || prm->strip_row0 % t2 ||
            prm->strip_row0 >= L || prm->strip_rows > L || prm->held_rows < prm->strip_rows + t2 ||
            prm->held_rows > L)
            return fail(OCT_EINVAL, "strip: strip_row0, strip_rows multiples of 2*By, strip_rows + 2*By <= "
                                    "held_rows <= L");
    }
    return OCT_OK;
}

bool is_strip(const oct_sim *s) { return s->strip_rows > 0; }

int whole_only(const oct_sim *s, const char *what) {
    return fail(OCT_EINVAL, std::string(what) + " needs a handle holding the whole lattice (this one holds a strip)");
}

void destroy_members(oct_sim *s) {
    if (s->own_lat && s->lat) cudaFree(s->lat);
    if (s->d_t) cudaFree(s->d_t);
    if (s->d_net) cudaFree(s->d_net);
    if (s->d_net_sum) cudaFree(s->d_net_sum);
    if (s->d_rows) cudaFree(s->d_rows);
    if (s->d_w2) cudaFree(s->d_w2);
    if (s->h_small) cudaFreeHost(s->h_small);
    if (s->snap) cudaFree(s->snap);
    if (s->d_ac_rows) cudaFree(s->d_ac_rows);
    if (s->d_ac) cudaFree(s->d_ac);
    for (cudaEvent_t e : s->ev)
        if (e) cudaEventDestroy(e);
    if (s->own_stream && s->stream) cudaStreamDestroy(s->stream);
}

int sim_create(const oct_params *prm, oct_sim **out) {
    int Bx, By, cx, cy;
    int rc = validate(prm, &Bx, &By, &cx, &cy);
    if (rc) return rc;
    oct_sim *s = new (std::nothrow) oct_sim();
    if (!s) return fail(OCT_ENOMEM, "host allocation of the handle failed");
    s->L = prm->L;
    s->p = prm->p;
    s->q = prm->q;
    s->seed = prm->seed;
    s->Bx = Bx;
    s->By = By;
    s->cx = cx;
    s->cy = cy;
    s->scheme = prm->scheme;
    s->strip_row0 = prm->strip_row0;
    s->strip_rows = prm->strip_rows;
    s->held_rows = prm->strip_rows ? prm->held_rows : 0;
    const int64_t plane_rows = is_strip(s) ? s->held_rows : s->L;
    cudaError_t e = cudaGetDevice(&s->device);
    const size_t lat_bytes = static_cast<size_t>(plane_rows) * static_cast<size_t>(s->L) / 4;
    if (e == cudaSuccess) {
        if (prm->stream) {
            s->stream = static_cast<cudaStream_t>(prm->stream);
        } else {
            e = cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking);
            s->own_stream = (e == cudaSuccess);
        }
    }
    if (e == cudaSuccess) {
        if (prm->lattice) {
            if (reinterpret_cast<uintptr_t>(prm->lattice) % 16u != 0u) {
                if (s->own_stream) cudaStreamDestroy(s->stream);
                delete s;
                return fail(OCT_EINVAL, "an external lattice buffer must be 16-byte aligned");
            }
            s->lat = static_cast<uint32_t *>(prm->lattice);
        } else {
            e = cudaMalloc(&s->lat, lat_bytes);
            s->own_lat = (e == cudaSuccess);
        }
    }
    if (e == cudaSuccess) e = cudaMalloc(&s->d_t, sizeof(uint32_t));
    if (e == cudaSuccess) e = cudaMalloc(&s->d_net, sizeof(unsigned long long) * 3 * oct::kNetSlots);
    if (e == cudaSuccess) e = cudaMalloc(&s->d_net_sum, 3 * sizeof(long long));
    if (e == cudaSuccess) e = cudaMalloc(&s->d_rows, sizeof(oct::W2RowSums) * s->L);
    if (e == cudaSuccess) e = cudaMalloc(&s->d_w2, sizeof(oct::W2Result));
    if (e == cudaSuccess) e = cudaMallocHost(&s->h_small, 256);
    if (e == cudaSuccess) e = cudaMemsetAsync(s->d_t, 0, sizeof(uint32_t), s->stream);
    if (e == cudaSuccess)
        e = cudaMemsetAsync(s->d_net, 0, sizeof(unsigned long long) * 3 * oct::kNetSlots, s->stream);
    if (e == cudaSuccess && !prm->no_init)
        e = oct::launch_init_flat_rows(s->lat, static_cast<uint32_t>(s->L), static_cast<uint32_t>(plane_rows), s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) {
        const bool oom = (e == cudaErrorMemoryAllocation);
        destroy_members(s);
        delete s;
        return oom ? fail(OCT_ENOMEM, "device allocation failed") : cuda_fail(e, "oct_create");
    }
    oct::StepArgs &a = s->args;
    a.lat = s->lat;
    a.L = static_cast<uint32_t>(s->L);
    a.wpr = static_cast<uint32_t>(s->L / 32);
    a.Bx = static_cast<uint32_t>(Bx);
    a.By = static_cast<uint32_t>(By);
    a.GX = static_cast<uint32_t>(Bx / 32);
    a.GY = static_cast<uint32_t>(By / 16);
    a.tiles_x = static_cast<uint32_t>(s->L / (2 * Bx));
    a.tiles_y = static_cast<uint32_t>(s->L / (2 * By));
    a.k0 = static_cast<uint32_t>(s->seed & 0xFFFFFFFFu);
    a.k1 = static_cast<uint32_t>(s->seed >> 32);
    const bool p_rand = s->p > 0.0 && s->p < 1.0, q_rand = s->q > 0.0 && s->q < 1.0;
    a.thr_p = p_rand ? threshold32(s->p) : 0u;
    a.thr_q = q_rand ? threshold32(s->q) : 0u;
    a.p_always = (s->p == 1.0) ? 0xFFFFFFFFu : 0u;
    a.q_always = (s->q == 1.0) ? 0xFFFFFFFFu : 0u;
    a.p_random = p_rand ? 0xFFFFFFFFu : 0u;
    a.q_random = q_rand ? 0xFFFFFFFFu : 0u;
    a.t_ptr = s->d_t;
    a.k = 0;
    a.net = s->d_net;
    a.draws = s->d_net + oct::kNetSlots;
    a.tails = s->d_net + 2 * oct::kNetSlots;
    s->any_random = p_rand || q_rand;
    // DB delays border attempts only when two neighbouring flips could meet
    // kernel variants: 0 DT, 1 DB with all attempts of a step together, 2 DB
    // with delayed borders (both rates non-zero), 3 DTrDTr
    a.scheme = (s->scheme == OCT_SCHEME_DB) ? ((s->p > 0.0 && s->q > 0.0) ? 2u : 1u)
               : (s->scheme == OCT_SCHEME_DTR) ? 3u : 0u;
    a.cx = static_cast<uint32_t>(cx);
    a.cy = static_cast<uint32_t>(cy);
    a.row0 = static_cast<uint32_t>(s->strip_row0);
    a.plane_rows = static_cast<uint32_t>(plane_rows);
    a.strip_tiles_y = is_strip(s) ? static_cast<uint32_t>(s->strip_rows / (2 * By)) : 0u;
    *out = s;
    return OCT_OK;
}

int set_time(oct_sim *s, int64_t t) {
    if (t < 0 || t > 0xFFFFFFFFll) return fail(OCT_EINVAL, "t must lie in [0, 2^32-1]");
    const uint32_t tt = static_cast<uint32_t>(t);
    OCT_CUDA(cudaMemcpyAsync(s->d_t, &tt, sizeof(tt), cudaMemcpyHostToDevice, s->stream));
    OCT_CUDA(cudaMemsetAsync(s->d_net, 0, sizeof(unsigned long long) * 3 * oct::kNetSlots, s->stream));
    OCT_CUDA(cudaStreamSynchronize(s->stream));
    s->t = static_cast<uint64_t>(t);
    s->next_k = 0;
    return OCT_OK;
}

// Words of the handle's planar buffer (both planes): the whole lattice, or the held rows of a strip.
size_t lattice_words(const oct_sim *s) {
    const int64_t rows = is_strip(s) ? s->held_rows : s->L;
    return static_cast<size_t>(rows) * static_cast<size_t>(s->L) / 16;
}

// Canonical rows per conversion chunk: at most 64 MiB of staging.
uint32_t canon_chunk_rows(const oct_sim *s) {
    const size_t row_bytes = static_cast<size_t>(s->L / 4) * 4;
    size_t rows = (size_t{64} << 20) / row_bytes;
    if (rows < 1) rows = 1;
    if (rows > static_cast<size_t>(s->L / 4)) rows = static_cast<size_t>(s->L / 4);
    return static_cast<uint32_t>(rows);
}

}  // namespace

extern "C" {

int oct_create(int64_t L, double p, double q, uint64_t seed, oct_sim **out) {
    if (!out) return fail(OCT_EINVAL, "out must not be NULL");
    oct_params prm;
    std::memset(&prm, 0, sizeof(prm));
    prm.L = L;
    prm.p = p;
    prm.q = q;
    prm.seed = seed;
    return sim_create(&prm, out);
}

int oct_create_ex(const oct_params *prm, oct_sim **out) {
    if (!prm || !out) return fail(OCT_EINVAL, "prm and out must not be NULL");
    return sim_create(prm, out);
}

int oct_run_mcs(oct_sim *s, int64_t n) {
    if (!s) return fail(OCT_EINVAL, "NULL handle");
    if (is_strip(s)) return whole_only(s, "oct_run_mcs (strips run oct_device_step between halo exchanges)");
    if (s->next_k != 0) return fail(OCT_EINVAL, "an MCS run by oct_device_step is not finished");
    if (n < 0) return fail(OCT_EINVAL, "n must be >= 0");
    if (s->t + static_cast<uint64_t>(n) > 0xFFFFFFFFull) return fail(OCT_EINVAL, "MCS counter would pass 2^32-1");
    OCT_CUDA(cudaSetDevice(s->device));
    for (int64_t i = 0; i < n; ++i) {
        for (uint32_t k = 0; k < 4; ++k) {
            s->args.k = k;
            if (s->timing) {
                if (s->ev_used == kEventPairs) {
                    int rc = flush_timing(s);
                    if (rc) return rc;
                }
                OCT_CUDA(cudaEventRecord(s->ev[2 * s->ev_used], s->stream));
            }
            OCT_CUDA(oct::launch_dtrdt_step(s->args, s->any_random, s->stream));
            if (s->timing) {
                OCT_CUDA(cudaEventRecord(s->ev[2 * s->ev_used + 1], s->stream));
                ++s->ev_used;
                ++s->step_launches;
            }
        }
        OCT_CUDA(oct::launch_advance_t(s->d_t, s->stream));
    }
    s->t += static_cast<uint64_t>(n);
    return OCT_OK;
}

int oct_device_step(oct_sim *s, int k) {
    if (!s) return fail(OCT_EINVAL, "NULL handle");
    if (k < 0 || k > 3) return fail(OCT_EINVAL, "device step k must lie in 0..3");
    if (k != s->next_k) return fail(OCT_EINVAL, "device steps must run in the order 0, 1, 2, 3 (then oct_end_mcs)");
    if (s->t >= 0xFFFFFFFFull) return fail(OCT_EINVAL, "MCS counter would pass 2^32-1");
    OCT_CUDA(cudaSetDevice(s->device));
    s->args.k = static_cast<uint32_t>(k);
    if (s->timing) {
        if (s->ev_used == kEventPairs) {
            int rc = flush_timing(s);
            if (rc) return rc;
        }
        OCT_CUDA(cudaEventRecord(s->ev[2 * s->ev_used], s->stream));
    }
    OCT_CUDA(oct::launch_dtrdt_step(s->args, s->any_random, s->stream));
    if (s->timing) {
        OCT_CUDA(cudaEventRecord(s->ev[2 * s->ev_used + 1], s->stream));
        ++s->ev_used;
        ++s->step_launches;
    }
    s->next_k = k + 1;
    return OCT_OK;
}

int oct_end_mcs(oct_sim *s) {
    if (!s) return fail(OCT_EINVAL, "NULL handle");
    if (s->next_k != 4) return fail(OCT_EINVAL, "oct_end_mcs needs device steps 0..3 first");
    OCT_CUDA(cudaSetDevice(s->device));
    OCT_CUDA(oct::launch_advance_t(s->d_t, s->stream));
    s->t += 1;
    s->next_k = 0;
    return OCT_OK;
}

int oct_mcs_draw(uint64_t seed, int64_t L, uint32_t t, int64_t *ox, int64_t *oy, int32_t perm[4]) {
    if (!ox || !oy || !perm) return fail(OCT_EINVAL, "NULL argument");
    if (L < 2 || L > (int64_t{1} << 20)) return fail(OCT_EINVAL, "L must lie in [2, 2^20]");
    const uint4 M = oct::philox4x32_10(t, 0u, 0u, oct::kTagMcs << 28, static_cast<uint32_t>(seed & 0xFFFFFFFFu),
                                       static_cast<uint32_t>(seed >> 32));
    *ox = static_cast<int64_t>((static_cast<uint64_t>(M.x) * static_cast<uint64_t>(L)) >> 32);
    *oy = static_cast<int64_t>((static_cast<uint64_t>(M.y) * static_cast<uint64_t>(L)) >> 32);
    // the (M.z * 24) >> 32 -th permutation of (0, 1, 2, 3) in lexicographic order
    uint32_t idx = static_cast<uint32_t>((static_cast<uint64_t>(M.z) * 24u) >> 32);
    int avail[4] = {0, 1, 2, 3}, n = 4;
    const uint32_t fact[4] = {6, 2, 1, 1};
    for (int i = 0; i < 4; ++i) {
        const uint32_t pick = idx / fact[i];
        idx %= fact[i];
        perm[i] = avail[pick];
        for (int j = static_cast<int>(pick); j < n - 1; ++j) avail[j] = avail[j + 1];
        --n;
    }
    return OCT_OK;
}

int oct_strip_measure(oct_sim *s, oct_strip_sums *out) {
    if (!s || !out) return fail(OCT_EINVAL, "NULL argument");
    if (!is_strip(s)) return fail(OCT_EINVAL, "oct_strip_measure needs a strip handle (use oct_measure_w2)");
    OCT_CUDA(cudaSetDevice(s->device));
    OCT_CUDA(oct::launch_net_sum(s->d_net, s->d_net + oct::kNetSlots, s->d_net + 2 * oct::kNetSlots,
                                 s->d_net_sum, s->stream));
    OCT_CUDA(oct::launch_w2_rows(s->lat, static_cast<uint32_t>(s->L), static_cast<uint32_t>(s->strip_rows),
                                 static_cast<uint32_t>(s->held_rows), s->d_rows, s->d_w2, s->stream));
    auto *res = static_cast<oct::W2Result *>(s->h_small);
    auto *net = reinterpret_cast<long long *>(static_cast<char *>(s->h_small) + 128);
    OCT_CUDA(cudaMemcpyAsync(res, s->d_w2, sizeof(oct::W2Result), cudaMemcpyDeviceToHost, s->stream));
    OCT_CUDA(cudaMemcpyAsync(net, s->d_net_sum, 3 * sizeof(long long), cudaMemcpyDeviceToHost, s->stream));
    OCT_CUDA(cudaStreamSynchronize(s->stream));
    out->rows = s->strip_rows;
    out->L = s->L;
    out->f = res->f0;
    out->e_last = res->e_last;
    out->p1 = res->s1;
    out->p2_lo = res->s2_lo;
    out->p2_hi = res->s2_hi;
    out->lo = res->lo;
    out->hi = res->hi;
    out->t = static_cast<int64_t>(s->t);
    out->net_flips = net[0];
    return OCT_OK;
}

int oct_strip_combine(const oct_strip_sums *parts, int64_t n, oct_w2 *out) {
    if (!parts || !out || n < 1) return fail(OCT_EINVAL, "need n >= 1 strips and an output");
    const int64_t L = parts[0].L;
    int64_t rows = 0;
    for (int64_t r = 0; r < n; ++r) {
        if (parts[r].L != L || parts[r].rows < 1 || parts[r].t != parts[0].t)
            return fail(OCT_EINVAL, "strips of one lattice at one time, in row order");
        rows += parts[r].rows;
    }
    if (rows != L) return fail(OCT_EINVAL, "the strips' rows must add up to L");
    __int128 S1 = 0, S2 = 0, B = 0;
    int64_t hmax = 0, net = 0;
    for (int64_t r = 0; r < n; ++r) {
        const oct_strip_sums &p = parts[r];
        if (r > 0) B += parts[r - 1].e_last + p.f;  // h(0, first row of strip r)
        const __int128 P2 = static_cast<__int128>((static_cast<unsigned __int128>(p.p2_hi) << 64) | p.p2_lo);
        const __int128 LH = static_cast<__int128>(L) * p.rows;
        S1 += LH * B + p.p1;
        S2 += LH * B * B + 2 * B * p.p1 + P2;
        const __int128 a = B + p.lo, b = B + p.hi;
        const __int128 m = std::max(a < 0 ? -a : a, b < 0 ? -b : b);
        hmax = std::max<int64_t>(hmax, static_cast<int64_t>(m));
        net += p.net_flips;
    }
    const __int128 N = static_cast<__int128>(L) * L;
    const __int128 num = N * S2 - S1 * S1;
    out->t = parts[0].t;
    out->n_sites = static_cast<int64_t>(N);
    out->s1 = static_cast<int64_t>(S1);
    out->s2_lo = static_cast<uint64_t>(static_cast<unsigned __int128>(S2));
    out->s2_hi = static_cast<uint64_t>(static_cast<unsigned __int128>(S2) >> 64);
    out->net_flips = net;
    out->hmax = hmax;
    out->w2 = static_cast<double>(num) / (static_cast<double>(N) * static_cast<double>(N));
    return OCT_OK;
}

namespace {

// Enqueues the W^2 reduction (Eq. (3)) and the copy of its sums into the
// handle's pinned staging area.
int enqueue_w2(oct_sim *s) {
    OCT_CUDA(oct::launch_net_sum(s->d_net, s->d_net + oct::kNetSlots, s->d_net + 2 * oct::kNetSlots,
                                 s->d_net_sum, s->stream));
    OCT_CUDA(oct::launch_w2(s->lat, static_cast<uint32_t>(s->L), s->d_rows, s->d_w2, s->stream));
    auto *res = static_cast<oct::W2Result *>(s->h_small);
    auto *net = reinterpret_cast<long long *>(static_cast<char *>(s->h_small) + 128);
    OCT_CUDA(cudaMemcpyAsync(res, s->d_w2, sizeof(oct::W2Result), cudaMemcpyDeviceToHost, s->stream));
    OCT_CUDA(cudaMemcpyAsync(net, s->d_net_sum, 2 * sizeof(long long), cudaMemcpyDeviceToHost, s->stream));
    s->w2_pending = true;
    s->w2_t = s->t;
    return OCT_OK;
}

// Waits for the enqueued measurement and forms W^2 = (N S2 - S1^2) / N^2 in
// 128-bit integers, one conversion to double at the end.
int finish_w2(oct_sim *s, oct_w2 *out) {
    s->w2_pending = false;
    OCT_CUDA(cudaStreamSynchronize(s->stream));
    const auto *res = static_cast<const oct::W2Result *>(s->h_small);
    const auto *net = reinterpret_cast<const long long *>(static_cast<const char *>(s->h_small) + 128);
    const __int128 N = static_cast<__int128>(s->L) * s->L;
    const __int128 S2 = static_cast<__int128>((static_cast<unsigned __int128>(res->s2_hi) << 64) | res->s2_lo);
    const __int128 num = N * S2 - static_cast<__int128>(res->s1) * res->s1;
    out->t = static_cast<int64_t>(s->w2_t);
    out->n_sites = static_cast<int64_t>(N);
    out->s1 = res->s1;
    out->s2_lo = res->s2_lo;
    out->s2_hi = res->s2_hi;
    out->net_flips = net[0];
    s->draws = net[1];
    out->hmax = res->hmax;
    out->w2 = static_cast<double>(num) / (static_cast<double>(N) * static_cast<double>(N));
    return OCT_OK;
}

}  // namespace

int oct_measure_w2(oct_sim *s, oct_w2 *out) {
    if (!s || !out) return fail(OCT_EINVAL, "NULL argument");
    if (is_strip(s)) return whole_only(s, "oct_measure_w2 (use oct_strip_measure)");
    if (s->w2_pending) return fail(OCT_EINVAL, "a measurement from oct_measure_w2_async is pending: call oct_w2_wait");
    OCT_CUDA(cudaSetDevice(s->device));
    const int rc = enqueue_w2(s);
    if (rc) return rc;
    return finish_w2(s, out);
}

int oct_measure_w2_async(oct_sim *s) {
    if (!s) return fail(OCT_EINVAL, "NULL argument");
    if (is_strip(s)) return whole_only(s, "oct_measure_w2_async");
    if (s->w2_pending) return fail(OCT_EINVAL, "a measurement is already pending: call oct_w2_wait");
    OCT_CUDA(cudaSetDevice(s->device));
    return enqueue_w2(s);
}

int oct_w2_wait(oct_sim *s, oct_w2 *out) {
    if (!s || !out) return fail(OCT_EINVAL, "NULL argument");
    if (!s->w2_pending) return fail(OCT_EINVAL, "no measurement pending (oct_measure_w2_async first)");
    OCT_CUDA(cudaSetDevice(s->device));
    return finish_w2(s, out);
}

int oct_get_lattice(oct_sim *s, uint32_t *host, size_t words) {
    if (!s || !host) return fail(OCT_EINVAL, "NULL argument");
    if (is_strip(s)) return whole_only(s, "oct_get_lattice");
    if (words != lattice_words(s)) return fail(OCT_EINVAL, "words must equal the buffer's words (L*L/16; held_rows*L/16 for a strip)");
    OCT_CUDA(cudaSetDevice(s->device));
    const uint32_t chunk = canon_chunk_rows(s), ncr = static_cast<uint32_t>(s->L / 4);
    const size_t row_words = static_cast<size_t>(s->L / 4);
    uint32_t *tmp = nullptr;
    OCT_CUDA(cudaMalloc(&tmp, chunk * row_words * 4));
    int rc = OCT_OK;
    for (uint32_t r = 0; r < ncr && rc == OCT_OK; r += chunk) {
        const uint32_t n = (ncr - r < chunk) ? ncr - r : chunk;
        cudaError_t e = oct::launch_pack_canonical(s->lat, static_cast<uint32_t>(s->L), r, n, tmp, s->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(host + r * row_words, tmp, n * row_words * 4, cudaMemcpyDeviceToHost, s->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
        if (e != cudaSuccess) rc = cuda_fail(e, "oct_get_lattice");
    }
    cudaFree(tmp);
    return rc;
}

int oct_set_lattice(oct_sim *s, const uint32_t *host, size_t words, int64_t t) {
    if (!s || !host) return fail(OCT_EINVAL, "NULL argument");
    if (is_strip(s)) return whole_only(s, "oct_set_lattice");
    if (words != lattice_words(s)) return fail(OCT_EINVAL, "words must equal the buffer's words (L*L/16; held_rows*L/16 for a strip)");
    if (t < 0 || t > 0xFFFFFFFFll) return fail(OCT_EINVAL, "t must lie in [0, 2^32-1]");
    OCT_CUDA(cudaSetDevice(s->device));
    const uint32_t chunk = canon_chunk_rows(s), ncr = static_cast<uint32_t>(s->L / 4);
    const size_t row_words = static_cast<size_t>(s->L / 4);
    uint32_t *tmp = nullptr;
    OCT_CUDA(cudaMalloc(&tmp, chunk * row_words * 4));
    int rc = OCT_OK;
    for (uint32_t r = 0; r < ncr && rc == OCT_OK; r += chunk) {
        const uint32_t n = (ncr - r < chunk) ? ncr - r : chunk;
        cudaError_t e = cudaMemcpyAsync(tmp, host + r * row_words, n * row_words * 4, cudaMemcpyHostToDevice, s->stream);
        if (e == cudaSuccess) e = oct::launch_unpack_canonical(tmp, static_cast<uint32_t>(s->L), r, n, s->lat, s->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
        if (e != cudaSuccess) rc = cuda_fail(e, "oct_set_lattice");
    }
    cudaFree(tmp);
    if (rc) return rc;
    return set_time(s, t);
}

int oct_get_planes(oct_sim *s, uint32_t *host, size_t words) {
    if (!s || !host) return fail(OCT_EINVAL, "NULL argument");
    if (words != lattice_words(s)) return fail(OCT_EINVAL, "words must equal the buffer's words (L*L/16; held_rows*L/16 for a strip)");
    OCT_CUDA(cudaSetDevice(s->device));
    OCT_CUDA(cudaMemcpyAsync(host, s->lat, words * 4, cudaMemcpyDeviceToHost, s->stream));
    OCT_CUDA(cudaStreamSynchronize(s->stream));
    return OCT_OK;
}

int oct_get_planes_async(oct_sim *s, uint32_t *host, size_t words) {
    if (!s || !host) return fail(OCT_EINVAL, "NULL argument");
    if (words != lattice_words(s)) return fail(OCT_EINVAL, "words must equal the buffer's words (L*L/16; held_rows*L/16 for a strip)");
    OCT_CUDA(cudaSetDevice(s->device));
    OCT_CUDA(cudaMemcpyAsync(host, s->lat, words * 4, cudaMemcpyDeviceToHost, s->stream));
    return OCT_OK;
}

int oct_set_planes(oct_sim *s, const uint32_t *host, size_t words, int64_t t) {
    if (!s || !host) return fail(OCT_EINVAL, "NULL argument");
    if (words != lattice_words(s)) return fail(OCT_EINVAL, "words must equal the buffer's words (L*L/16; held_rows*L/16 for a strip)");
    if (t < 0 || t > 0xFFFFFFFFll) return fail(OCT_EINVAL, "t must lie in [0, 2^32-1]");
    OCT_CUDA(cudaSetDevice(s->device));
    OCT_CUDA(cudaMemcpyAsync(s->lat, host, words * 4, cudaMemcpyHostToDevice, s->stream));
    return set_time(s, t);
}

int oct_get_window(oct_sim *s, int64_t wx, int64_t wy, int64_t W, int64_t H, uint8_t *X, uint8_t *Y) {
    if (!s || !X || !Y) return fail(OCT_EINVAL, "NULL argument");
    if (is_strip(s)) return whole_only(s, "oct_get_window");
    const int64_t L = s->L;
    if (W < 1 || H < 1 || W > L || H > L) return fail(OCT_EINVAL, "window must satisfy 1 <= W, H <= L");
    OCT_CUDA(cudaSetDevice(s->device));
    const int64_t wpr = L / 32;
    wx = ((wx % L) + L) % L;
    wy = ((wy % L) + L) % L;
    std::vector<uint32_t> rows(static_cast<size_t>(H) * wpr * 2);
    // copy whole rows of both planes, at most two contiguous row ranges per plane
    for (int plane = 0; plane < 2; ++plane) {
        int64_t done = 0;
        while (done < H) {
            const int64_t y = (wy + done) % L;
            const int64_t n = (L - y < H - done) ? L - y : H - done;
            const uint32_t *src = s->lat + static_cast<size_t>(plane) * L * wpr + static_cast<size_t>(y) * wpr;
            OCT_CUDA(cudaMemcpyAsync(rows.data() + (static_cast<size_t>(plane) * H + done) * wpr, src,
                                     static_cast<size_t>(n) * wpr * 4, cudaMemcpyDeviceToHost, s->stream));
            done += n;
        }
    }
    OCT_CUDA(cudaStreamSynchronize(s->stream));
    for (int64_t j = 0; j < H; ++j)
        for (int64_t i = 0; i < W; ++i) {
            const int64_t x = (wx + i) % L;
            const uint32_t xw = rows[static_cast<size_t>(j) * wpr + x / 32];
            const uint32_t yw = rows[(static_cast<size_t>(H) + j) * wpr + x / 32];
            X[j * W + i] = static_cast<uint8_t>((xw >> (x % 32)) & 1u);
            Y[j * W + i] = static_cast<uint8_t>((yw >> (x % 32)) & 1u);
        }
    return OCT_OK;
}

int oct_get_info(oct_sim *s, oct_info *out) {
    if (!s || !out) return fail(OCT_EINVAL, "NULL argument");
    out->L = s->L;
    out->t = static_cast<int64_t>(s->t);
    out->Bx = s->Bx;
    out->By = s->By;
    out->cx = s->cx;
    out->cy = s->cy;
    out->p = s->p;
    out->q = s->q;
    out->seed = s->seed;
    out->stream = s->stream;
    out->lattice = s->lat;
    out->lattice_bytes = static_cast<int64_t>(lattice_words(s) * 4);
    out->scheme = s->scheme;
    out->reserved = 0;
    return OCT_OK;
}

int oct_sync(oct_sim *s) {
    if (!s) return fail(OCT_EINVAL, "NULL handle");
    OCT_CUDA(cudaSetDevice(s->device));
    OCT_CUDA(cudaStreamSynchronize(s->stream));
    return OCT_OK;
}

int oct_set_timing(oct_sim *s, int enable) {
    if (!s) return fail(OCT_EINVAL, "NULL handle");
    OCT_CUDA(cudaSetDevice(s->device));
    if (s->ev.empty()) {
        s->ev.resize(2 * kEventPairs);
        for (auto &e : s->ev) OCT_CUDA(cudaEventCreate(&e));
    }
    int rc = flush_timing(s);
    if (rc) return rc;
    s->timing = enable != 0;
    s->step_ms = 0.0;
    s->step_launches = 0;
    return OCT_OK;
}

int oct_get_timing(oct_sim *s, double *step_ms, int64_t *step_launches, double *other_ms) {
    if (!s) return fail(OCT_EINVAL, "NULL handle");
    int rc = flush_timing(s);
    if (rc) return rc;
    if (step_ms) *step_ms = s->step_ms;
    if (step_launches) *step_launches = s->step_launches;
    if (other_ms) *other_ms = 0.0;
    return OCT_OK;
}

int oct_destroy(oct_sim *s) {
    if (!s) return OCT_OK;
    cudaSetDevice(s->device);
    if (s->stream) cudaStreamSynchronize(s->stream);
    destroy_members(s);
    delete s;
    return OCT_OK;
}



int oct_snapshot(oct_sim *s) {
    if (!s) return fail(OCT_EINVAL, "NULL argument");
    if (is_strip(s)) return whole_only(s, "oct_snapshot");
    OCT_CUDA(cudaSetDevice(s->device));
    const size_t bytes = lattice_words(s) * 4;
    if (!s->snap) {
        OCT_CUDA(cudaMalloc(&s->snap, bytes));
        OCT_CUDA(cudaMalloc(&s->d_ac_rows, static_cast<size_t>(s->L) * sizeof(oct::AcRowSums)));
        OCT_CUDA(cudaMalloc(&s->d_ac, sizeof(oct::AcResult)));
    }
    OCT_CUDA(cudaMemcpyAsync(s->snap, s->lat, bytes, cudaMemcpyDeviceToDevice, s->stream));
    s->snap_t = static_cast<int64_t>(s->t);
    return OCT_OK;
}

int oct_measure_ac(oct_sim *s, oct_ac *out) {
    if (!s || !out) return fail(OCT_EINVAL, "NULL argument");
    if (!s->snap) return fail(OCT_EINVAL, "no snapshot: call oct_snapshot first");
    OCT_CUDA(cudaSetDevice(s->device));
    OCT_CUDA(oct::launch_two_time(s->lat, s->snap, static_cast<uint32_t>(s->L), s->d_ac_rows, s->d_ac,
                                  s->stream));
    oct::AcResult r{};
    OCT_CUDA(cudaMemcpyAsync(&r, s->d_ac, sizeof(r), cudaMemcpyDeviceToHost, s->stream));
    OCT_CUDA(cudaStreamSynchronize(s->stream));
    oct::fill_ac(s->L, r, out);
    out->t = static_cast<int64_t>(s->t);
    out->s = s->snap_t;
    return OCT_OK;
}

int oct_two_time_planes(const void *lat_t, const void *lat_s, int64_t L, void *stream, oct_ac *out) {
    if (!lat_t || !lat_s || !out) return fail(OCT_EINVAL, "NULL argument");
    if (L < 32 || L > (1 << 20) || L % 32 != 0) return fail(OCT_EINVAL, "L must be a multiple of 32 in [32, 2^20]");
    cudaStream_t st = stream ? static_cast<cudaStream_t>(stream) : cudaStreamLegacy;
    void *scratch = nullptr;
    const size_t rows_bytes = static_cast<size_t>(L) * sizeof(oct::AcRowSums);
    OCT_CUDA(cudaMallocAsync(&scratch, rows_bytes + sizeof(oct::AcResult), st));
    auto *rows = static_cast<oct::AcRowSums *>(scratch);
    auto *res = reinterpret_cast<oct::AcResult *>(static_cast<char *>(scratch) + rows_bytes);
    oct::AcResult r{};
    cudaError_t e = oct::launch_two_time(static_cast<const uint32_t *>(lat_t), static_cast<const uint32_t *>(lat_s),
                                         static_cast<uint32_t>(L), rows, res, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&r, res, sizeof(r), cudaMemcpyDeviceToHost, st);
    const cudaError_t ef = cudaFreeAsync(scratch, st);
    if (e == cudaSuccess) e = ef;
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "oct_two_time_planes");
    oct::fill_ac(L, r, out);
    out->t = -1;
    out->s = -1;
    return OCT_OK;
}

int oct_get_stats(oct_sim *s, oct_stats *out) {
    if (!s || !out) return fail(OCT_EINVAL, "NULL argument");
    OCT_CUDA(cudaSetDevice(s->device));
    OCT_CUDA(oct::launch_net_sum(s->d_net, s->d_net + oct::kNetSlots, s->d_net + 2 * oct::kNetSlots,
                                 s->d_net_sum, s->stream));
    auto *net = reinterpret_cast<long long *>(static_cast<char *>(s->h_small) + 192);
    OCT_CUDA(cudaMemcpyAsync(net, s->d_net_sum, 3 * sizeof(long long), cudaMemcpyDeviceToHost, s->stream));
    OCT_CUDA(cudaStreamSynchronize(s->stream));
    out->t = static_cast<int64_t>(s->t);
    out->net_flips = net[0];
    out->draws = net[1];
    out->tail_blocks = net[2];
    return OCT_OK;
}

int oct_probe_int_rate(int op, double *ops_per_clk_per_sm, double *sm_mhz, int *sm_count) {
    if (!ops_per_clk_per_sm || !sm_mhz || (op != 0 && op != 1)) return fail(OCT_EINVAL, "bad probe arguments");
    int dev = 0, sms = 0;
    OCT_CUDA(cudaGetDevice(&dev));
    OCT_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    OCT_CUDA(oct::measure_int_rate(op, sms, ops_per_clk_per_sm, sm_mhz));
    if (sm_count) *sm_count = sms;
    return OCT_OK;
}

const char *oct_strerror(int code) {
    switch (code) {
        case OCT_OK: return "success";
        case OCT_EINVAL: return "invalid argument";
        case OCT_ENOMEM: return "out of memory";
        case OCT_ECUDA: return "CUDA runtime error";
        case OCT_ETIMEDOUT: return "bounded device wait timed out";
        case OCT_EINTERNAL: return "internal consistency check failed";
        case OCT_EUNSUPPORTED: return "unsupported configuration";
        default: return "unknown error code";
    }
}

const char *oct_last_error(void) { return g_last_error.c_str(); }

}  // extern "C"
