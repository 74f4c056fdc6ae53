// Batched DTrDT: many independent realizations (replicas) of different L, p, q
// advanced together, one device step of every replica per launch.
//
// Each replica is its own DTrDT simulation (its own key, origin, set order
// and lattice; Sec. 3 / 3.1); batching changes only how the work reaches the
// GPU.  The device-step work of all replicas is a list of (replica, device
// tile) items.  A replica whose sub-tile holds G lane groups of 32 x 16
// sites (G = 8 for 64 x 64 sub-tiles, 2 for 32 x 32) takes G consecutive
// lanes, so one warp carries 32/G sub-tiles, possibly of different replicas.
// Items are bucketed by G and by acceptance mode and packed into warp
// descriptors; persistent warps claim descriptors from an atomic queue.
// Because the sub-tiles of one warp draw their own block-level sets, the
// collective step takes the set per lane (step_candidates_rt / step_apply_rt);
// sub-tiles of 32 groups fill a warp alone and take the uniform path.  All
// replicas advance in lock step: one MCS is four device steps, each one launch
// per acceptance mode and warp kind, captured once in a CUDA graph and
// replayed.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "../../include/oct.h"
#include "oct_internal.h"
#include "subtile.cuh"

namespace oct {
namespace {

struct ReplicaDev {
    uint32_t *lat;
    unsigned long long *counters;  // [net flips, acceptance draws]
    uint32_t L, wpr, Bx, By, GX, GY, tiles_x, tiles_y;
    uint32_t k0, k1, thr_p, thr_q;
    uint32_t p_always, q_always, p_random, q_random;
};

struct BatchItem {
    uint32_t rep;
    uint32_t T;
};

struct WarpDesc {
    uint32_t first;  // first item
    uint32_t n;      // items in this warp (32 / G at most)
    uint32_t G;      // lanes per item
    uint32_t GX;     // lane columns per item
};

constexpr int kBatchWarps = 4;
constexpr int kBatchBlocksPerSM = 4;

// LANE_SETS: the warp holds several sub-tiles (fewer than 32 groups each), each
// with its own set draws; otherwise one sub-tile fills the warp and the step
// takes the uniform row-offset path of the plain kernel.
// SCHEME: 0 DTrDT, 4 with deposition only (p = 1, q = 0), 5 with both rates
// strictly inside (0, 1) (the step variants of the plain kernel).
template <bool RANDOM, bool LANE_SETS, int SCHEME>
__global__ void __launch_bounds__(kBatchWarps * 32, kBatchBlocksPerSM)
    batch_step_kernel(const ReplicaDev *reps, const BatchItem *items, const WarpDesc *descs,
                      uint32_t n_descs, const uint32_t *t_of, uint32_t k, uint32_t *queue) {
    __shared__ __align__(16) uint32_t ring[kBatchWarps * 32 * kRingWordsPerLane];
    const int lane = threadIdx.x & 31;
    for (;;) {
        uint32_t di = 0;
        if (lane == 0) di = atomicAdd(queue, 1u);
        di = __shfl_sync(kFull, di, 0);
        if (di >= n_descs) break;  // the whole warp leaves together
        const WarpDesc wd = descs[di];
        const int G = static_cast<int>(wd.G);
        const int slot = lane / G, sub = lane % G;
        const bool active = slot < static_cast<int>(wd.n);
        const BatchItem it = items[wd.first + (active ? slot : 0)];
        const ReplicaDev R = reps[it.rep];
        const uint32_t t = t_of[it.rep];  // this replica's MCS index
        const uint32_t L = R.L;
        const uint4 M = philox4x32_10(t, 0u, 0u, kTagMcs << 28, R.k0, R.k1);
        const uint32_t ox = static_cast<uint32_t>((static_cast<uint64_t>(M.x) * L) >> 32);
        const uint32_t oy = static_cast<uint32_t>((static_cast<uint64_t>(M.y) * L) >> 32);
        const uint32_t pidx = static_cast<uint32_t>((static_cast<uint64_t>(M.z) * 24u) >> 32);
        const int sigma = perm_element(pidx, k);
        const uint32_t tx = it.T % R.tiles_x, ty = it.T / R.tiles_x;
        const uint32_t x0 = static_cast<uint32_t>(
            (static_cast<uint64_t>(ox) + 2ull * R.Bx * tx + static_cast<uint64_t>(R.Bx) * (sigma & 1)) % L);
        const uint32_t y0 = static_cast<uint32_t>(
            (static_cast<uint64_t>(oy) + 2ull * R.By * ty + static_cast<uint64_t>(R.By) * (sigma >> 1)) % L);
        LaneCtx c;
        c.GX = static_cast<int>(wd.GX);
        c.GY = G / c.GX;
        c.gx = sub % c.GX;
        c.gy = sub / c.GX;
        c.active = active;
        c.last = lane | (G - 1);
        c.t = t;
        c.k = k;
        c.T = it.T;
        c.g = static_cast<uint32_t>(sub);
        c.k0 = R.k0;
        c.k1 = R.k1;
        c.thr_p = R.thr_p;
        c.thr_q = R.thr_q;
        c.p_always = R.p_always;
        c.q_always = R.q_always;
        c.p_random = R.p_random;
        c.q_random = R.q_random;
        int net = 0, draws = 0, tails = 0;
        run_subtile<RANDOM, LANE_SETS, SCHEME>(R.lat, L, L, R.wpr, R.Bx, R.By, x0, y0, active, c,
                                  ring + ((threadIdx.x >> 5) * 32 + (lane & ~(G - 1))) * kRingWordsPerLane,
                                  net, draws, tails);
        // sum over the G lanes of the item (items start at multiples of G)
        for (int o = G >> 1; o > 0; o >>= 1) {
            net += __shfl_xor_sync(kFull, net, o);
            draws += __shfl_xor_sync(kFull, draws, o);
        }
        if (active && sub == 0) {
            if (net != 0)
                atomicAdd(&R.counters[0], static_cast<unsigned long long>(static_cast<long long>(net)));
            if (RANDOM && draws != 0) atomicAdd(&R.counters[1], static_cast<unsigned long long>(draws));
        }
    }
}

// Advances the MCS counter of every active replica.
__global__ void batch_advance_kernel(uint32_t *t_of, const uint32_t *active, uint32_t n_active) {
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n_active; i += gridDim.x * blockDim.x)
        t_of[active[i]] += 1u;
}

}  // namespace
}  // namespace oct

namespace {

constexpr int kModes = 4;
constexpr int kKinds = 2 * kModes;  // acceptance mode x (several sub-tiles per warp, or one)
// Each kind's replicas are split into up to kParts parts of about equal
// sites, each of at least kMinPartSites sites; a branch (kind, part) is the
// unit of the captured graph (see enqueue_mcs).
constexpr int kParts = 3;
constexpr uint64_t kMinPartSites = uint64_t{1} << 26;
constexpr int kBranches = kKinds * kParts;

int bfail(int code, const std::string &msg) {
    oct::set_last_error(msg);
    return code;
}

#define BATCH_CUDA(call)                                                                  \
    do {                                                                                  \
        cudaError_t e_ = (call);                                                          \
        if (e_ != cudaSuccess) return bfail(OCT_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

uint32_t thr32(double p) { return static_cast<uint32_t>(std::floor(std::ldexp(p, 32))); }

}  // namespace

namespace oct {
namespace {

// One of the two alternating copies of the work list (replica table, items,
// warp descriptors, active slots).  A rebuild fills the copy the running work
// does not read, from pinned staging memory, in stream order: no host wait.
struct WorkBuf {
    ReplicaDev *reps = nullptr;
    size_t reps_cap = 0;
    BatchItem *items = nullptr;
    size_t items_cap = 0;
    WarpDesc *descs = nullptr;
    size_t descs_cap = 0;
    uint32_t *active = nullptr;
    size_t active_cap = 0;
    char *host = nullptr;     // pinned staging of the last copy into this set
    size_t host_cap = 0;
    cudaEvent_t copied = nullptr;  // recorded after that copy
};

// An asynchronous W^2 measurement: the exact sums, the replica's counters and
// its time, copied to pinned host memory behind an event.
struct MeasureRecord {
    W2Result res;
    unsigned long long cnt[2];
    uint32_t t;
    uint32_t pad[3];
};
constexpr int kMeasureRing = 1024;
constexpr int kMarkRing = 64;
constexpr int kGraphMcs = 4;  // MCS in the batch's longer captured graph

}  // namespace
}  // namespace oct

struct oct_batch {
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    cudaMemPool_t pool = nullptr;     // replica lattices, stream-ordered
    // slots (a replica keeps its slot until removed)
    std::vector<oct_replica> reps;
    std::vector<uint32_t *> lat;      // per slot, nullptr if free
    std::vector<char> used;
    std::vector<int64_t> free_slots;
    size_t capacity = 0;
    uint32_t *d_t = nullptr;            // capacity MCS counters
    unsigned long long *counters = nullptr;  // 2 * capacity: net flips, draws
    // work list of the current membership
    bool dirty = true;
    oct::WorkBuf wb[2];
    int cur = 0;  // the copy the enqueued work reads
    uint32_t n_active = 0;
    // work lists by kind = 2 * mode + (one sub-tile per warp); modes: 0 no
    // acceptance draws, 1 draws, 2 draws for both rates, 3 deposition only
    // work lists by branch = kParts * kind + part
    uint32_t n_desc[kBranches] = {};
    uint32_t desc_first[kBranches] = {};
    // the active replicas ordered by branch: act_n[br] of them from act_first[br]
    uint32_t act_first[kBranches] = {};
    uint32_t act_n[kBranches] = {};
    uint32_t *d_queue = nullptr;  // 4 * kBranches counters: (device step, branch)
    oct::W2RowSums *d_rows = nullptr;
    int64_t rows_cap = 0;
    oct::W2Result *d_w2 = nullptr;
    void *h_small = nullptr;
    // two-time autocorrelations: per slot, the lattice at its waiting time
    std::vector<uint32_t *> snap;
    std::vector<int64_t> snap_t;
    oct::AcRowSums *d_ac_rows = nullptr;
    int64_t ac_rows_cap = 0;
    oct::AcResult *d_ac = nullptr;
    uint64_t ticks = 0;  // MCS run by oct_batch_run
    int grid = 0;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;        // one MCS
    cudaGraph_t graph_n = nullptr;
    cudaGraphExec_t exec_n = nullptr;      // kGraphMcs MCS
    // side streams and events of the captured MCS: one branch per kind
    cudaStream_t side[kBranches] = {};
    cudaEvent_t fork_ev = nullptr;
    cudaEvent_t join_ev[kBranches] = {};
    // asynchronous measurements: a ring of records (device and pinned host)
    oct::MeasureRecord *d_req = nullptr;
    oct::MeasureRecord *h_req = nullptr;
    std::vector<cudaEvent_t> req_ev;
    std::vector<int64_t> req_L;
    int64_t req_next = 0;  // tickets handed out so far
    // stream marks (oct_batch_mark): a ring of events
    std::vector<cudaEvent_t> mark_ev;
    int64_t mark_next = 0;  // marks handed out so far
    bool timing = false;
    std::vector<cudaEvent_t> ev;
    int ev_used = 0;
    double step_ms = 0.0;
    int64_t step_launches = 0;
};

namespace {

void drop_graph(oct_batch *b) {
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    if (b->exec_n) cudaGraphExecDestroy(b->exec_n);
    if (b->graph_n) cudaGraphDestroy(b->graph_n);
    b->exec = nullptr;
    b->graph = nullptr;
    b->exec_n = nullptr;
    b->graph_n = nullptr;
}

void batch_free(oct_batch *b) {
    drop_graph(b);
    for (uint32_t *p : b->lat)
        if (p) cudaFreeAsync(p, b->stream);
    for (uint32_t *p : b->snap)
        if (p) cudaFreeAsync(p, b->stream);
    if (b->stream) cudaStreamSynchronize(b->stream);
    cudaFree(b->d_ac_rows);
    cudaFree(b->d_ac);
    cudaFree(b->d_t);
    cudaFree(b->counters);
    for (oct::WorkBuf &w : b->wb) {
        cudaFree(w.reps);
        cudaFree(w.items);
        cudaFree(w.descs);
        cudaFree(w.active);
        if (w.host) cudaFreeHost(w.host);
        if (w.copied) cudaEventDestroy(w.copied);
    }
    cudaFree(b->d_req);
    if (b->h_req) cudaFreeHost(b->h_req);
    for (cudaEvent_t e : b->req_ev)
        if (e) cudaEventDestroy(e);  // ring events are created on first use
    for (cudaEvent_t e : b->mark_ev)
        if (e) cudaEventDestroy(e);
    cudaFree(b->d_queue);
    for (int br = 0; br < kBranches; ++br) {
        if (b->side[br]) cudaStreamDestroy(b->side[br]);
        if (b->join_ev[br]) cudaEventDestroy(b->join_ev[br]);
    }
    if (b->fork_ev) cudaEventDestroy(b->fork_ev);
    cudaFree(b->d_rows);
    cudaFree(b->d_w2);
    if (b->h_small) cudaFreeHost(b->h_small);
    for (cudaEvent_t e : b->ev)
        if (e) cudaEventDestroy(e);
    if (b->pool) cudaMemPoolDestroy(b->pool);
    if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
}

int check_replica(oct_replica &R) {
    if (R.L < 64 || R.L > 16384 || R.L % 64) return bfail(OCT_EINVAL, "replica L must be a multiple of 64 in [64, 16384]");
    if (!(R.p >= 0.0 && R.p <= 1.0 && R.q >= 0.0 && R.q <= 1.0))
        return bfail(OCT_EINVAL, "replica p and q must lie in [0, 1]");
    if (R.Bx == 0 && R.By == 0) {
        R.Bx = (R.L % 128 == 0) ? 64 : 32;
        R.By = R.Bx;
    }
    const int GX = R.Bx / 32, GY = R.By / 16, G = GX * GY;
    if (R.Bx < 32 || R.By < 16 || R.Bx % 32 || R.By % 16 || R.L % (2 * R.Bx) || R.L % (2 * R.By) ||
        (GX & (GX - 1)) || (GY & (GY - 1)) || G > 32)
        return bfail(OCT_EINVAL, "replica sub-tile must be a power-of-two number (at most 32) of "
                                 "32x16-site groups in each direction and divide L/2");
    return OCT_OK;
}

oct::ReplicaDev replica_dev(const oct_batch *b, int64_t slot) {
    const oct_replica &R = b->reps[slot];
    oct::ReplicaDev D;
    D.lat = b->lat[slot];
    D.counters = b->counters + 2 * slot;
    D.L = static_cast<uint32_t>(R.L);
    D.wpr = static_cast<uint32_t>(R.L / 32);
    D.Bx = static_cast<uint32_t>(R.Bx);
    D.By = static_cast<uint32_t>(R.By);
    D.GX = static_cast<uint32_t>(R.Bx / 32);
    D.GY = static_cast<uint32_t>(R.By / 16);
    D.tiles_x = static_cast<uint32_t>(R.L / (2 * R.Bx));
    D.tiles_y = static_cast<uint32_t>(R.L / (2 * R.By));
    D.k0 = static_cast<uint32_t>(R.seed & 0xFFFFFFFFu);
    D.k1 = static_cast<uint32_t>(R.seed >> 32);
    const bool pr = R.p > 0.0 && R.p < 1.0, qr = R.q > 0.0 && R.q < 1.0;
    D.thr_p = pr ? thr32(R.p) : 0u;
    D.thr_q = qr ? thr32(R.q) : 0u;
    D.p_always = (R.p == 1.0) ? 0xFFFFFFFFu : 0u;
    D.q_always = (R.q == 1.0) ? 0xFFFFFFFFu : 0u;
    D.p_random = pr ? 0xFFFFFFFFu : 0u;
    D.q_random = qr ? 0xFFFFFFFFu : 0u;
    return D;
}

template <typename T>
cudaError_t ensure(T **p, size_t *cap, size_t need, cudaStream_t st) {
    if (need <= *cap) return cudaSuccess;
    size_t n = std::max<size_t>(need, 2 * *cap);
    // stream-ordered: work already enqueued may still read the old buffer
    if (*p) {
        cudaError_t e = cudaFreeAsync(*p, st);
        if (e != cudaSuccess) return e;
    }
    *p = nullptr;
    *cap = 0;
    cudaError_t e = cudaMallocAsync(reinterpret_cast<void **>(p), sizeof(T) * n, st);
    if (e == cudaSuccess) *cap = n;
    return e;
}

// Grows the per-slot tables, keeping the device-resident counters.
cudaError_t grow_slots(oct_batch *b, size_t need) {
    if (need <= b->capacity) return cudaSuccess;
    const size_t n = std::max<size_t>(need, std::max<size_t>(64, 2 * b->capacity));
    uint32_t *t = nullptr;
    unsigned long long *c = nullptr;
    cudaError_t e = cudaStreamSynchronize(b->stream);
    if (e == cudaSuccess) e = cudaMalloc(&t, sizeof(uint32_t) * n);
    if (e == cudaSuccess) e = cudaMalloc(&c, sizeof(unsigned long long) * 2 * n);
    if (e == cudaSuccess && b->capacity) {
        e = cudaMemcpy(t, b->d_t, sizeof(uint32_t) * b->capacity, cudaMemcpyDeviceToDevice);
        if (e == cudaSuccess)
            e = cudaMemcpy(c, b->counters, sizeof(unsigned long long) * 2 * b->capacity, cudaMemcpyDeviceToDevice);
    }
    if (e != cudaSuccess) {
        cudaFree(t);
        cudaFree(c);
        return e;
    }
    cudaFree(b->d_t);
    cudaFree(b->counters);
    b->d_t = t;
    b->counters = c;
    b->capacity = n;
    b->dirty = true;
    return cudaSuccess;
}

// Rebuilds the replica table and the warp work list of the active replicas
// into the work-list copy the enqueued work does not read, by asynchronous
// copies on the batch's stream (the host waits only for the staging memory of
// the copy before last, long finished).
cudaError_t rebuild(oct_batch *b) {
    cudaError_t e = cudaSuccess;
    drop_graph(b);  // an executable graph still running is freed when it completes
    std::vector<oct::ReplicaDev> rd(b->capacity);
    // replicas by kind, then each kind split into up to kParts parts of about
    // equal sites (largest first, each to the lightest part)
    std::vector<uint32_t> by_kind[kKinds];
    for (size_t slot = 0; slot < b->reps.size(); ++slot) {
        if (!b->used[slot]) continue;
        rd[slot] = replica_dev(b, static_cast<int64_t>(slot));
        const oct::ReplicaDev &D = rd[slot];
        const int mode = (D.p_random && D.q_random) ? 2
                         : (D.p_random || D.q_random) ? 1
                         : (D.p_always && !D.q_always) ? 3 : 0;
        by_kind[2 * mode + (D.GX * D.GY == 32u ? 1 : 0)].push_back(static_cast<uint32_t>(slot));
    }
    std::vector<uint32_t> by_branch[kBranches];
    for (int kind = 0; kind < kKinds; ++kind) {
        std::vector<uint32_t> &v = by_kind[kind];
        std::stable_sort(v.begin(), v.end(), [&](uint32_t a, uint32_t c) { return rd[a].L > rd[c].L; });
        uint64_t sites = 0;
        for (uint32_t slot : v) sites += static_cast<uint64_t>(rd[slot].L) * rd[slot].L;
        const int parts = static_cast<int>(std::max<uint64_t>(1, std::min<uint64_t>(kParts, sites / kMinPartSites)));
        uint64_t load[kParts] = {};
        for (uint32_t slot : v) {
            int part = 0;
            for (int q = 1; q < parts; ++q)
                if (load[q] < load[part]) part = q;
            load[part] += static_cast<uint64_t>(rd[slot].L) * rd[slot].L;
            by_branch[kind * kParts + part].push_back(slot);
        }
    }
    std::vector<uint32_t> active;
    std::vector<oct::BatchItem> items;
    std::vector<oct::WarpDesc> descs;
    for (int br = 0; br < kBranches; ++br) {
        b->act_first[br] = static_cast<uint32_t>(active.size());
        b->act_n[br] = static_cast<uint32_t>(by_branch[br].size());
        active.insert(active.end(), by_branch[br].begin(), by_branch[br].end());
        // the branch's items bucketed by lane layout, then packed into warps
        std::vector<oct::BatchItem> bucket[6][6];
        for (uint32_t slot : by_branch[br]) {
            const oct::ReplicaDev &D = rd[slot];
            int gxi = 0, gyi = 0;
            while ((1u << gxi) < D.GX) ++gxi;
            while ((1u << gyi) < D.GY) ++gyi;
            for (uint32_t T = 0; T < D.tiles_x * D.tiles_y; ++T) bucket[gxi][gyi].push_back({slot, T});
        }
        b->desc_first[br] = static_cast<uint32_t>(descs.size());
        for (int gxi = 5; gxi >= 0; --gxi)
            for (int gyi = 5; gyi >= 0; --gyi) {
                const uint32_t GX = 1u << gxi, G = GX << gyi;
                if (G > 32u) continue;
                const uint32_t per = 32u / G;
                auto &bk = bucket[gxi][gyi];
                for (size_t i = 0; i < bk.size(); i += per) {
                    oct::WarpDesc d;
                    d.first = static_cast<uint32_t>(items.size());
                    d.n = static_cast<uint32_t>(std::min<size_t>(per, bk.size() - i));
                    d.G = G;
                    d.GX = GX;
                    for (uint32_t j = 0; j < d.n; ++j) items.push_back(bk[i + j]);
                    descs.push_back(d);
                }
            }
        b->n_desc[br] = static_cast<uint32_t>(descs.size()) - b->desc_first[br];
    }
    const int nxt = 1 - b->cur;
    oct::WorkBuf &w = b->wb[nxt];
    const size_t n_reps = std::max<size_t>(1, b->capacity);
    e = ensure(&w.reps, &w.reps_cap, n_reps, b->stream);
    if (e == cudaSuccess) e = ensure(&w.items, &w.items_cap, std::max<size_t>(1, items.size()), b->stream);
    if (e == cudaSuccess) e = ensure(&w.descs, &w.descs_cap, std::max<size_t>(1, descs.size()), b->stream);
    if (e == cudaSuccess) e = ensure(&w.active, &w.active_cap, std::max<size_t>(1, active.size()), b->stream);
    // pinned staging: reps, items, descs, active back to back (16-byte aligned parts)
    auto up16 = [](size_t v) { return (v + 15) & ~static_cast<size_t>(15); };
    const size_t o_items = up16(sizeof(oct::ReplicaDev) * b->capacity);
    const size_t o_descs = o_items + up16(sizeof(oct::BatchItem) * items.size());
    const size_t o_active = o_descs + up16(sizeof(oct::WarpDesc) * descs.size());
    const size_t bytes = std::max<size_t>(16, o_active + sizeof(uint32_t) * active.size());
    if (e == cudaSuccess && w.copied) e = cudaEventSynchronize(w.copied);  // its last copy has left the staging
    if (e == cudaSuccess && bytes > w.host_cap) {
        if (w.host) cudaFreeHost(w.host);
        w.host = nullptr;
        w.host_cap = 0;
        e = cudaMallocHost(reinterpret_cast<void **>(&w.host), 2 * bytes);
        if (e == cudaSuccess) w.host_cap = 2 * bytes;
    }
    if (e == cudaSuccess && !w.copied) e = cudaEventCreateWithFlags(&w.copied, cudaEventDisableTiming);
    if (e != cudaSuccess) return e;
    if (b->capacity) std::memcpy(w.host, rd.data(), sizeof(oct::ReplicaDev) * b->capacity);
    if (!items.empty()) std::memcpy(w.host + o_items, items.data(), sizeof(oct::BatchItem) * items.size());
    if (!descs.empty()) std::memcpy(w.host + o_descs, descs.data(), sizeof(oct::WarpDesc) * descs.size());
    if (!active.empty()) std::memcpy(w.host + o_active, active.data(), sizeof(uint32_t) * active.size());
    if (b->capacity)
        e = cudaMemcpyAsync(w.reps, w.host, sizeof(oct::ReplicaDev) * b->capacity, cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess && !items.empty())
        e = cudaMemcpyAsync(w.items, w.host + o_items, sizeof(oct::BatchItem) * items.size(), cudaMemcpyHostToDevice,
                            b->stream);
    if (e == cudaSuccess && !descs.empty())
        e = cudaMemcpyAsync(w.descs, w.host + o_descs, sizeof(oct::WarpDesc) * descs.size(), cudaMemcpyHostToDevice,
                            b->stream);
    if (e == cudaSuccess && !active.empty())
        e = cudaMemcpyAsync(w.active, w.host + o_active, sizeof(uint32_t) * active.size(), cudaMemcpyHostToDevice,
                            b->stream);
    if (e == cudaSuccess) e = cudaEventRecord(w.copied, b->stream);
    if (e != cudaSuccess) return e;
    b->cur = nxt;
    b->n_active = static_cast<uint32_t>(active.size());
    b->dirty = false;
    return cudaSuccess;
}

// Enqueues device step k of the current MCS of the replicas of one branch.
cudaError_t enqueue_branch_step(oct_batch *b, uint32_t k, int br, cudaStream_t st) {
    uint32_t *q = b->d_queue + kBranches * k + br;
    cudaError_t e = cudaMemsetAsync(q, 0, sizeof(uint32_t), st);
    if (e != cudaSuccess) return e;
    const oct::WorkBuf &w = b->wb[b->cur];
    const oct::WarpDesc *descs = w.descs + b->desc_first[br];
    const uint32_t nd = b->n_desc[br];
    const int kind = br / kParts;
    const int blocks = std::min<int>(b->grid, static_cast<int>((nd + oct::kBatchWarps - 1) / oct::kBatchWarps));
    const dim3 grid(blocks), block(oct::kBatchWarps * 32);
#define OCT_BATCH(R, LS, SC) \
    oct::batch_step_kernel<R, LS, SC><<<grid, block, 0, st>>>(w.reps, w.items, descs, nd, b->d_t, k, q)
    switch (kind) {
        case 0: OCT_BATCH(false, true, 0); break;
        case 1: OCT_BATCH(false, false, 0); break;
        case 2: OCT_BATCH(true, true, 0); break;
        case 3: OCT_BATCH(true, false, 0); break;
        case 4: OCT_BATCH(true, true, 5); break;
        case 5: OCT_BATCH(true, false, 5); break;
        case 6: OCT_BATCH(false, true, 4); break;
        default: OCT_BATCH(false, false, 4); break;
    }
#undef OCT_BATCH
    return cudaGetLastError();
}

// Enqueues device step k of the current MCS of every active replica, branch by branch.
cudaError_t enqueue_step(oct_batch *b, uint32_t k, cudaStream_t st) {
    for (int br = 0; br < kBranches; ++br) {
        if (b->n_desc[br] == 0) continue;
        cudaError_t e = enqueue_branch_step(b, k, br, st);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t enqueue_advance(oct_batch *b, cudaStream_t st) {
    if (b->n_active == 0) return cudaSuccess;
    const int blocks = static_cast<int>(std::min<uint32_t>(1024u, (b->n_active + 255u) / 256u));
    oct::batch_advance_kernel<<<blocks, 256, 0, st>>>(b->d_t, b->wb[b->cur].active, b->n_active);
    return cudaGetLastError();
}

// Advances the MCS counters of the replicas of one branch.
cudaError_t enqueue_advance_branch(oct_batch *b, int br, cudaStream_t st) {
    const uint32_t n = b->act_n[br];
    if (n == 0) return cudaSuccess;
    const int blocks = static_cast<int>(std::min<uint32_t>(1024u, (n + 255u) / 256u));
    oct::batch_advance_kernel<<<blocks, 256, 0, st>>>(b->d_t, b->wb[b->cur].active + b->act_first[br], n);
    return cudaGetLastError();
}

// nmcs MCS for capture on st.  The replicas of different branches (kinds,
// and parts of a kind) share no memory and no counter, so each branch's
// device steps and its own MCS-counter advances form a branch of the graph
// (forked from st on a side stream and joined back at the end); the branches
// run concurrently, so one branch's launches fill the device while another's
// drain, and over several MCS no branch waits for the others at MCS
// boundaries.
cudaError_t enqueue_mcs(oct_batch *b, cudaStream_t st, int nmcs) {
    cudaError_t e = cudaSuccess;
    if (!b->fork_ev) e = cudaEventCreateWithFlags(&b->fork_ev, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventRecord(b->fork_ev, st);
    for (int br = 0; br < kBranches && e == cudaSuccess; ++br) {
        if (b->n_desc[br] == 0) continue;
        if (!b->side[br]) e = cudaStreamCreateWithFlags(&b->side[br], cudaStreamNonBlocking);
        if (e == cudaSuccess && !b->join_ev[br]) e = cudaEventCreateWithFlags(&b->join_ev[br], cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(b->side[br], b->fork_ev, 0);
        for (int i = 0; i < nmcs && e == cudaSuccess; ++i) {
            for (uint32_t k = 0; k < 4 && e == cudaSuccess; ++k) e = enqueue_branch_step(b, k, br, b->side[br]);
            if (e == cudaSuccess) e = enqueue_advance_branch(b, br, b->side[br]);
        }
        if (e == cudaSuccess) e = cudaEventRecord(b->join_ev[br], b->side[br]);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(st, b->join_ev[br], 0);
    }
    return e;
}

// Captures nmcs MCS of the current membership into *graph / *exec.
cudaError_t capture_mcs(oct_batch *b, int nmcs, cudaGraph_t *graph, cudaGraphExec_t *exec) {
    cudaStream_t cap = nullptr;
    cudaError_t e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
    if (e != cudaSuccess) return e;
    e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        const cudaError_t e2 = enqueue_mcs(b, cap, nmcs);
        e = cudaStreamEndCapture(cap, graph);
        if (e == cudaSuccess) e = e2;
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(exec, *graph, 0);
    cudaStreamDestroy(cap);
    return e;
}

int flush_batch_timing(oct_batch *b) {
    if (b->ev_used == 0) return OCT_OK;
    BATCH_CUDA(cudaEventSynchronize(b->ev[2 * (b->ev_used - 1) + 1]));
    for (int i = 0; i < b->ev_used; ++i) {
        float ms = 0.f;
        BATCH_CUDA(cudaEventElapsedTime(&ms, b->ev[2 * i], b->ev[2 * i + 1]));
        b->step_ms += ms;
    }
    b->ev_used = 0;
    return OCT_OK;
}

bool valid_slot(const oct_batch *b, int64_t slot) {
    return slot >= 0 && slot < static_cast<int64_t>(b->reps.size()) && b->used[slot];
}

int add_replica(oct_batch *b, const oct_replica *in, int64_t *slot_out) {
    oct_replica R = *in;
    int rc = check_replica(R);
    if (rc) return rc;
    int64_t slot;
    if (!b->free_slots.empty()) {
        slot = b->free_slots.back();
        b->free_slots.pop_back();
    } else {
        slot = static_cast<int64_t>(b->reps.size());
        BATCH_CUDA(grow_slots(b, static_cast<size_t>(slot) + 1));
        b->reps.emplace_back();
        b->lat.push_back(nullptr);
        b->used.push_back(0);
        b->snap.push_back(nullptr);
        b->snap_t.push_back(-1);
    }
    const size_t bytes = static_cast<size_t>(R.L) * R.L / 4;
    uint32_t *p = nullptr;
    cudaError_t e = cudaMallocFromPoolAsync(reinterpret_cast<void **>(&p), bytes, b->pool, b->stream);
    if (e != cudaSuccess) {
        b->free_slots.push_back(slot);
        return e == cudaErrorMemoryAllocation ? bfail(OCT_ENOMEM, "no device memory for the replica lattice")
                                              : bfail(OCT_ECUDA, std::string("cudaMallocFromPoolAsync: ") + cudaGetErrorString(e));
    }
    b->reps[slot] = R;
    b->lat[slot] = p;
    b->used[slot] = 1;
    BATCH_CUDA(oct::launch_init_flat(p, static_cast<uint32_t>(R.L), b->stream));
    BATCH_CUDA(cudaMemsetAsync(b->d_t + slot, 0, sizeof(uint32_t), b->stream));
    BATCH_CUDA(cudaMemsetAsync(b->counters + 2 * slot, 0, 2 * sizeof(unsigned long long), b->stream));
    b->dirty = true;
    if (slot_out) *slot_out = slot;
    return OCT_OK;
}

int measure_slot(oct_batch *b, int64_t slot, oct_w2 *out) {
    const int64_t L = b->reps[slot].L;
    if (L > b->rows_cap) {
        cudaFree(b->d_rows);
        b->d_rows = nullptr;
        b->rows_cap = 0;
        BATCH_CUDA(cudaMalloc(&b->d_rows, sizeof(oct::W2RowSums) * L));
        b->rows_cap = L;
    }
    auto *res = static_cast<oct::W2Result *>(b->h_small);
    auto *cnt = reinterpret_cast<unsigned long long *>(static_cast<char *>(b->h_small) + 64);
    auto *tt = reinterpret_cast<uint32_t *>(static_cast<char *>(b->h_small) + 96);
    BATCH_CUDA(oct::launch_w2(b->lat[slot], static_cast<uint32_t>(L), b->d_rows, b->d_w2, b->stream));
    BATCH_CUDA(cudaMemcpyAsync(res, b->d_w2, sizeof(oct::W2Result), cudaMemcpyDeviceToHost, b->stream));
    BATCH_CUDA(cudaMemcpyAsync(cnt, b->counters + 2 * slot, 2 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, b->stream));
    BATCH_CUDA(cudaMemcpyAsync(tt, b->d_t + slot, sizeof(uint32_t), cudaMemcpyDeviceToHost, b->stream));
    BATCH_CUDA(cudaStreamSynchronize(b->stream));
    const __int128 N = static_cast<__int128>(L) * L;
    const __int128 S2 = static_cast<__int128>((static_cast<unsigned __int128>(res->s2_hi) << 64) | res->s2_lo);
    const __int128 num = N * S2 - static_cast<__int128>(res->s1) * res->s1;
    out->t = static_cast<int64_t>(*tt);
    out->n_sites = static_cast<int64_t>(N);
    out->s1 = res->s1;
    out->s2_lo = res->s2_lo;
    out->s2_hi = res->s2_hi;
    out->net_flips = static_cast<int64_t>(cnt[0]);
    out->hmax = res->hmax;
    out->w2 = static_cast<double>(num) / (static_cast<double>(N) * static_cast<double>(N));
    return OCT_OK;
}

// W^2 from an asynchronous measurement record (numerator in 128-bit integers).
void record_to_w2(const oct::MeasureRecord &r, int64_t L, oct_w2 *out) {
    const __int128 N = static_cast<__int128>(L) * L;
    const __int128 S2 = static_cast<__int128>((static_cast<unsigned __int128>(r.res.s2_hi) << 64) | r.res.s2_lo);
    const __int128 num = N * S2 - static_cast<__int128>(r.res.s1) * r.res.s1;
    out->t = static_cast<int64_t>(r.t);
    out->n_sites = static_cast<int64_t>(N);
    out->s1 = r.res.s1;
    out->s2_lo = r.res.s2_lo;
    out->s2_hi = r.res.s2_hi;
    out->net_flips = static_cast<int64_t>(r.cnt[0]);
    out->hmax = r.res.hmax;
    out->w2 = static_cast<double>(num) / (static_cast<double>(N) * static_cast<double>(N));
}

int ticket_index(oct_batch *b, int64_t ticket, int *idx) {
    if (ticket < 0 || ticket >= b->req_next || ticket < b->req_next - oct::kMeasureRing)
        return bfail(OCT_EINVAL, "unknown or expired measurement ticket");
    *idx = static_cast<int>(ticket % oct::kMeasureRing);
    return OCT_OK;
}

}  // namespace

extern "C" {

int oct_batch_measure_async(oct_batch *b, int64_t slot, int64_t *ticket) {
    if (!b || !ticket || !valid_slot(b, slot)) return bfail(OCT_EINVAL, "no replica in that slot");
    BATCH_CUDA(cudaSetDevice(b->device));
    const int64_t L = b->reps[slot].L;
    if (!b->d_req) {
        BATCH_CUDA(cudaMalloc(&b->d_req, sizeof(oct::MeasureRecord) * oct::kMeasureRing));
        BATCH_CUDA(cudaMallocHost(&b->h_req, sizeof(oct::MeasureRecord) * oct::kMeasureRing));
        b->req_ev.assign(oct::kMeasureRing, nullptr);
        b->req_L.assign(oct::kMeasureRing, 0);
    }
    const int i = static_cast<int>(b->req_next % oct::kMeasureRing);
    if (b->req_ev[i]) {
        BATCH_CUDA(cudaEventSynchronize(b->req_ev[i]));  // the ring wrapped: the oldest record is done
    } else {
        BATCH_CUDA(cudaEventCreateWithFlags(&b->req_ev[i], cudaEventDisableTiming));
    }
    if (L > b->rows_cap) {  // stream-ordered: an earlier measurement may still use the old rows
        if (b->d_rows) BATCH_CUDA(cudaFreeAsync(b->d_rows, b->stream));
        b->d_rows = nullptr;
        b->rows_cap = 0;
        BATCH_CUDA(cudaMallocAsync(reinterpret_cast<void **>(&b->d_rows), sizeof(oct::W2RowSums) * L, b->stream));
        b->rows_cap = L;
    }
    oct::MeasureRecord *d = b->d_req + i;
    BATCH_CUDA(oct::launch_w2(b->lat[slot], static_cast<uint32_t>(L), b->d_rows, &d->res, b->stream));
    BATCH_CUDA(cudaMemcpyAsync(d->cnt, b->counters + 2 * slot, 2 * sizeof(unsigned long long),
                               cudaMemcpyDeviceToDevice, b->stream));
    BATCH_CUDA(cudaMemcpyAsync(&d->t, b->d_t + slot, sizeof(uint32_t), cudaMemcpyDeviceToDevice, b->stream));
    BATCH_CUDA(cudaMemcpyAsync(b->h_req + i, d, sizeof(oct::MeasureRecord), cudaMemcpyDeviceToHost, b->stream));
    BATCH_CUDA(cudaEventRecord(b->req_ev[i], b->stream));
    b->req_L[i] = L;
    *ticket = b->req_next++;
    return OCT_OK;
}

int oct_batch_poll(oct_batch *b, int64_t ticket, oct_w2 *out, int *ready) {
    if (!b || !out || !ready) return bfail(OCT_EINVAL, "NULL argument");
    int i = 0;
    int rc = ticket_index(b, ticket, &i);
    if (rc) return rc;
    BATCH_CUDA(cudaSetDevice(b->device));
    const cudaError_t e = cudaEventQuery(b->req_ev[i]);
    if (e == cudaErrorNotReady) {
        (void)cudaGetLastError();  // "not ready" is an answer, not an error: do not leave it behind
        *ready = 0;
        return OCT_OK;
    }
    if (e != cudaSuccess) return bfail(OCT_ECUDA, std::string("oct_batch_poll: ") + cudaGetErrorString(e));
    record_to_w2(b->h_req[i], b->req_L[i], out);
    *ready = 1;
    return OCT_OK;
}

int oct_batch_wait(oct_batch *b, int64_t ticket, oct_w2 *out) {
    if (!b || !out) return bfail(OCT_EINVAL, "NULL argument");
    int i = 0;
    int rc = ticket_index(b, ticket, &i);
    if (rc) return rc;
    BATCH_CUDA(cudaSetDevice(b->device));
    BATCH_CUDA(cudaEventSynchronize(b->req_ev[i]));
    record_to_w2(b->h_req[i], b->req_L[i], out);
    return OCT_OK;
}

int oct_replica_seed(uint64_t master_seed, uint32_t r, uint64_t *seed) {
    if (!seed) return bfail(OCT_EINVAL, "seed must not be NULL");
    const uint4 w = oct::philox4x32_10(r, 0u, 0u, oct::kTagReplica << 28,
                                       static_cast<uint32_t>(master_seed & 0xFFFFFFFFu),
                                       static_cast<uint32_t>(master_seed >> 32));
    *seed = static_cast<uint64_t>(w.x) | (static_cast<uint64_t>(w.y) << 32);
    return OCT_OK;
}

int oct_batch_create(int64_t n, const oct_replica *reps, void *stream, oct_batch **out) {
    if (n < 0 || (n > 0 && !reps) || !out) return bfail(OCT_EINVAL, "need n >= 0 replicas and non-NULL arrays");
    for (int64_t r = 0; r < n; ++r) {
        oct_replica R = reps[r];
        int rc = check_replica(R);
        if (rc) return rc;
    }
    oct_batch *b = new (std::nothrow) oct_batch();
    if (!b) return bfail(OCT_ENOMEM, "host allocation failed");
    cudaError_t e = cudaGetDevice(&b->device);
    if (e == cudaSuccess) {
        if (stream) {
            b->stream = static_cast<cudaStream_t>(stream);
        } else {
            e = cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking);
            b->own_stream = (e == cudaSuccess);
        }
    }
    if (e == cudaSuccess) {
        cudaMemPoolProps props;
        std::memset(&props, 0, sizeof(props));
        props.allocType = cudaMemAllocationTypePinned;
        props.handleTypes = cudaMemHandleTypeNone;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = b->device;
        e = cudaMemPoolCreate(&b->pool, &props);
        if (e == cudaSuccess) {
            uint64_t keep = ~uint64_t{0};  // keep freed lattices in the pool for reuse
            e = cudaMemPoolSetAttribute(b->pool, cudaMemPoolAttrReleaseThreshold, &keep);
        }
    }
    if (e == cudaSuccess) e = cudaMalloc(&b->d_queue, sizeof(uint32_t) * 4 * kBranches);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_w2, sizeof(oct::W2Result));
    if (e == cudaSuccess) e = cudaMallocHost(&b->h_small, 256);
    if (e == cudaSuccess) {
        int sms = 0;
        e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, b->device);
        b->grid = sms * oct::kBatchBlocksPerSM;
    }
    if (e == cudaSuccess) e = grow_slots(b, static_cast<size_t>(std::max<int64_t>(n, 1)));
    if (e != cudaSuccess) {
        const bool oom = (e == cudaErrorMemoryAllocation);
        batch_free(b);
        delete b;
        return oom ? bfail(OCT_ENOMEM, "device allocation failed")
                   : bfail(OCT_ECUDA, std::string("oct_batch_create: ") + cudaGetErrorString(e));
    }
    for (int64_t r = 0; r < n; ++r) {
        int rc = add_replica(b, &reps[r], nullptr);
        if (rc) {
            batch_free(b);
            delete b;
            return rc;
        }
    }
    if (cudaStreamSynchronize(b->stream) != cudaSuccess) {
        batch_free(b);
        delete b;
        return bfail(OCT_ECUDA, "oct_batch_create: initialisation failed");
    }
    *out = b;
    return OCT_OK;
}

int oct_batch_add(oct_batch *b, const oct_replica *r, int64_t *slot) {
    if (!b || !r) return bfail(OCT_EINVAL, "NULL argument");
    BATCH_CUDA(cudaSetDevice(b->device));
    return add_replica(b, r, slot);
}

int oct_batch_remove(oct_batch *b, int64_t slot) {
    if (!b || !valid_slot(b, slot)) return bfail(OCT_EINVAL, "no replica in that slot");
    BATCH_CUDA(cudaSetDevice(b->device));
    BATCH_CUDA(cudaFreeAsync(b->lat[slot], b->stream));
    b->lat[slot] = nullptr;
    if (b->snap[slot]) {
        BATCH_CUDA(cudaFreeAsync(b->snap[slot], b->stream));
        b->snap[slot] = nullptr;
    }
    b->snap_t[slot] = -1;
    b->used[slot] = 0;
    b->free_slots.push_back(slot);
    b->dirty = true;
    return OCT_OK;
}

int oct_batch_run(oct_batch *b, int64_t n) {
    if (!b) return bfail(OCT_EINVAL, "NULL batch");
    if (n < 0) return bfail(OCT_EINVAL, "bad MCS count");
    BATCH_CUDA(cudaSetDevice(b->device));
    if (b->dirty) BATCH_CUDA(rebuild(b));
    if (b->n_active == 0 || n == 0) {
        b->ticks += static_cast<uint64_t>(n);
        return OCT_OK;
    }
    if (b->timing) {
        // launch by launch, each device step bracketed by events
        for (int64_t i = 0; i < n; ++i) {
            for (uint32_t k = 0; k < 4; ++k) {
                if (b->ev_used == 256) {
                    int rc = flush_batch_timing(b);
                    if (rc) return rc;
                }
                BATCH_CUDA(cudaEventRecord(b->ev[2 * b->ev_used], b->stream));
                BATCH_CUDA(enqueue_step(b, k, b->stream));
                BATCH_CUDA(cudaEventRecord(b->ev[2 * b->ev_used + 1], b->stream));
                ++b->ev_used;
                ++b->step_launches;
            }
            BATCH_CUDA(enqueue_advance(b, b->stream));
        }
    } else {
        // kGraphMcs MCS per graph launch while that many are left, then one
        // at a time; each graph is captured on a private stream on first use
        // after a membership change and replayed on the batch's stream
        int64_t left = n;
        if (left >= oct::kGraphMcs) {
            if (!b->exec_n) {
                const cudaError_t e = capture_mcs(b, oct::kGraphMcs, &b->graph_n, &b->exec_n);
                if (e != cudaSuccess) return bfail(OCT_ECUDA, std::string("graph capture: ") + cudaGetErrorString(e));
            }
            for (; left >= oct::kGraphMcs; left -= oct::kGraphMcs) BATCH_CUDA(cudaGraphLaunch(b->exec_n, b->stream));
        }
        if (left > 0) {
            if (!b->exec) {
                const cudaError_t e = capture_mcs(b, 1, &b->graph, &b->exec);
                if (e != cudaSuccess) return bfail(OCT_ECUDA, std::string("graph capture: ") + cudaGetErrorString(e));
            }
            for (; left > 0; --left) BATCH_CUDA(cudaGraphLaunch(b->exec, b->stream));
        }
    }
    b->ticks += static_cast<uint64_t>(n);
    return OCT_OK;
}

int oct_batch_measure_w2(oct_batch *b, oct_w2 *out, int64_t n) {
    if (!b || !out || n != static_cast<int64_t>(b->reps.size()))
        return bfail(OCT_EINVAL, "out must hold one entry per slot");
    BATCH_CUDA(cudaSetDevice(b->device));
    for (int64_t slot = 0; slot < n; ++slot) {
        if (!b->used[slot]) {
            std::memset(&out[slot], 0, sizeof(oct_w2));
            continue;
        }
        int rc = measure_slot(b, slot, &out[slot]);
        if (rc) return rc;
    }
    return OCT_OK;
}

int oct_batch_measure_slot(oct_batch *b, int64_t slot, oct_w2 *out) {
    if (!b || !out || !valid_slot(b, slot)) return bfail(OCT_EINVAL, "no replica in that slot");
    BATCH_CUDA(cudaSetDevice(b->device));
    return measure_slot(b, slot, out);
}

int oct_batch_snapshot(oct_batch *b, int64_t slot) {
    if (!b || !valid_slot(b, slot)) return bfail(OCT_EINVAL, "no replica in that slot");
    BATCH_CUDA(cudaSetDevice(b->device));
    const int64_t L = b->reps[slot].L;
    const size_t bytes = static_cast<size_t>(L) * L / 4;
    if (!b->snap[slot]) {
        uint32_t *p = nullptr;
        cudaError_t e = cudaMallocFromPoolAsync(reinterpret_cast<void **>(&p), bytes, b->pool, b->stream);
        if (e != cudaSuccess)
            return e == cudaErrorMemoryAllocation ? bfail(OCT_ENOMEM, "no device memory for the snapshot")
                                                  : bfail(OCT_ECUDA, std::string("cudaMallocFromPoolAsync: ") + cudaGetErrorString(e));
        b->snap[slot] = p;
    }
    BATCH_CUDA(cudaMemcpyAsync(b->snap[slot], b->lat[slot], bytes, cudaMemcpyDeviceToDevice, b->stream));
    auto *tt = reinterpret_cast<uint32_t *>(static_cast<char *>(b->h_small) + 96);
    BATCH_CUDA(cudaMemcpyAsync(tt, b->d_t + slot, sizeof(uint32_t), cudaMemcpyDeviceToHost, b->stream));
    BATCH_CUDA(cudaStreamSynchronize(b->stream));
    b->snap_t[slot] = static_cast<int64_t>(*tt);
    return OCT_OK;
}

int oct_batch_measure_ac(oct_batch *b, int64_t slot, oct_ac *out) {
    if (!b || !out || !valid_slot(b, slot)) return bfail(OCT_EINVAL, "no replica in that slot");
    if (!b->snap[slot]) return bfail(OCT_EINVAL, "no snapshot in that slot: call oct_batch_snapshot first");
    BATCH_CUDA(cudaSetDevice(b->device));
    const int64_t L = b->reps[slot].L;
    if (L > b->ac_rows_cap) {
        cudaFree(b->d_ac_rows);
        b->d_ac_rows = nullptr;
        b->ac_rows_cap = 0;
        BATCH_CUDA(cudaMalloc(&b->d_ac_rows, sizeof(oct::AcRowSums) * L));
        b->ac_rows_cap = L;
    }
    if (!b->d_ac) BATCH_CUDA(cudaMalloc(&b->d_ac, sizeof(oct::AcResult)));
    BATCH_CUDA(oct::launch_two_time(b->lat[slot], b->snap[slot], static_cast<uint32_t>(L), b->d_ac_rows, b->d_ac,
                                    b->stream));
    oct::AcResult r{};
    BATCH_CUDA(cudaMemcpyAsync(&r, b->d_ac, sizeof(r), cudaMemcpyDeviceToHost, b->stream));
    auto *tt = reinterpret_cast<uint32_t *>(static_cast<char *>(b->h_small) + 96);
    BATCH_CUDA(cudaMemcpyAsync(tt, b->d_t + slot, sizeof(uint32_t), cudaMemcpyDeviceToHost, b->stream));
    BATCH_CUDA(cudaStreamSynchronize(b->stream));
    oct::fill_ac(L, r, out);
    out->t = static_cast<int64_t>(*tt);
    out->s = b->snap_t[slot];
    return OCT_OK;
}

int oct_batch_get_planes(oct_batch *b, int64_t slot, uint32_t *host, size_t words) {
    if (!b || !host || !valid_slot(b, slot)) return bfail(OCT_EINVAL, "no replica in that slot");
    const int64_t L = b->reps[slot].L;
    if (words != static_cast<size_t>(L) * L / 16) return bfail(OCT_EINVAL, "words must equal L*L/16");
    BATCH_CUDA(cudaSetDevice(b->device));
    BATCH_CUDA(cudaMemcpyAsync(host, b->lat[slot], words * 4, cudaMemcpyDeviceToHost, b->stream));
    BATCH_CUDA(cudaStreamSynchronize(b->stream));
    return OCT_OK;
}

int oct_batch_get_stats(oct_batch *b, int64_t *ticks, int64_t *n_active, int64_t *active_sites, int64_t *draws) {
    if (!b) return bfail(OCT_EINVAL, "NULL batch");
    BATCH_CUDA(cudaSetDevice(b->device));
    int64_t sites = 0, na = 0;
    for (size_t s = 0; s < b->reps.size(); ++s)
        if (b->used[s]) {
            sites += b->reps[s].L * b->reps[s].L;
            ++na;
        }
    if (ticks) *ticks = static_cast<int64_t>(b->ticks);
    if (n_active) *n_active = na;
    if (active_sites) *active_sites = sites;
    if (draws) {
        std::vector<unsigned long long> cnt(2 * b->reps.size());
        if (!cnt.empty()) {
            BATCH_CUDA(cudaMemcpyAsync(cnt.data(), b->counters, sizeof(unsigned long long) * cnt.size(),
                                       cudaMemcpyDeviceToHost, b->stream));
            BATCH_CUDA(cudaStreamSynchronize(b->stream));
        }
        int64_t d = 0;
        for (size_t s = 0; s < b->reps.size(); ++s)
            if (b->used[s]) d += static_cast<int64_t>(cnt[2 * s + 1]);
        *draws = d;
    }
    return OCT_OK;
}

int oct_batch_sync(oct_batch *b) {
    if (!b) return bfail(OCT_EINVAL, "NULL batch");
    BATCH_CUDA(cudaSetDevice(b->device));
    BATCH_CUDA(cudaStreamSynchronize(b->stream));
    return OCT_OK;
}

int oct_batch_mark(oct_batch *b, int64_t *mark) {
    if (!b || !mark) return bfail(OCT_EINVAL, "NULL argument");
    BATCH_CUDA(cudaSetDevice(b->device));
    if (b->mark_ev.empty()) b->mark_ev.assign(oct::kMarkRing, nullptr);
    const int i = static_cast<int>(b->mark_next % oct::kMarkRing);
    if (b->mark_ev[i]) {
        // the ring wrapped: the mark recorded here kMarkRing marks ago is passed first
        BATCH_CUDA(cudaEventSynchronize(b->mark_ev[i]));
    } else {
        BATCH_CUDA(cudaEventCreateWithFlags(&b->mark_ev[i], cudaEventDisableTiming));
    }
    BATCH_CUDA(cudaEventRecord(b->mark_ev[i], b->stream));
    *mark = b->mark_next++;
    return OCT_OK;
}

int oct_batch_mark_done(oct_batch *b, int64_t mark, int *done) {
    if (!b || !done) return bfail(OCT_EINVAL, "NULL argument");
    if (mark < 0 || mark >= b->mark_next) return bfail(OCT_EINVAL, "unknown stream mark");
    if (mark < b->mark_next - oct::kMarkRing) {  // its event was reused after the device passed it
        *done = 1;
        return OCT_OK;
    }
    BATCH_CUDA(cudaSetDevice(b->device));
    const cudaError_t e = cudaEventQuery(b->mark_ev[mark % oct::kMarkRing]);
    if (e == cudaErrorNotReady) {
        (void)cudaGetLastError();
        *done = 0;
        return OCT_OK;
    }
    if (e != cudaSuccess) return bfail(OCT_ECUDA, std::string("oct_batch_mark_done: ") + cudaGetErrorString(e));
    *done = 1;
    return OCT_OK;
}

int oct_batch_mark_wait(oct_batch *b, int64_t mark) {
    if (!b) return bfail(OCT_EINVAL, "NULL batch");
    if (mark < 0 || mark >= b->mark_next) return bfail(OCT_EINVAL, "unknown stream mark");
    if (mark < b->mark_next - oct::kMarkRing) return OCT_OK;
    BATCH_CUDA(cudaSetDevice(b->device));
    BATCH_CUDA(cudaEventSynchronize(b->mark_ev[mark % oct::kMarkRing]));
    return OCT_OK;
}

int oct_batch_set_timing(oct_batch *b, int enable) {
    if (!b) return bfail(OCT_EINVAL, "NULL batch");
    BATCH_CUDA(cudaSetDevice(b->device));
    if (b->ev.empty()) {
        b->ev.resize(512);
        for (auto &e : b->ev) BATCH_CUDA(cudaEventCreate(&e));
    }
    int rc = flush_batch_timing(b);
    if (rc) return rc;
    b->timing = enable != 0;
    b->step_ms = 0.0;
    b->step_launches = 0;
    return OCT_OK;
}

int oct_batch_get_timing(oct_batch *b, double *step_ms, int64_t *step_launches) {
    if (!b) return bfail(OCT_EINVAL, "NULL batch");
    int rc = flush_batch_timing(b);
    if (rc) return rc;
    if (step_ms) *step_ms = b->step_ms;
    if (step_launches) *step_launches = b->step_launches;
    return OCT_OK;
}

int oct_batch_destroy(oct_batch *b) {
    if (!b) return OCT_OK;
    cudaSetDevice(b->device);
    if (b->stream) cudaStreamSynchronize(b->stream);
    batch_free(b);
    delete b;
    return OCT_OK;
}

}  // extern "C"
