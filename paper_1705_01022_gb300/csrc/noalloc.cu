// oct_w2_noalloc: exact roughness of a caller's lattice without any allocation.
//
// Some callers cannot allocate device memory at the moment they want a
// roughness value: a host framework or plugin that owns all device memory and
// hands this library only a buffer and a stream, or a latency-critical loop in
// which cudaMalloc/cudaFree are not allowed because they can synchronise the
// device and stall other work.  For them this entry point runs the same
// roughness kernels as oct_measure_w2, but keeps their scratch (per-row partial
// sums and the 32-byte result block) in a fixed array compiled into the
// library instead of in handle-owned allocations.
//
// The array below is file-scope device memory: every GPU that loads the
// library holds kScratchBytes of it until the process exits.  Host code must
// not use the symbol itself as a device address; the address is fetched once
// per device with cudaGetSymbolAddress while that device is current.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "../../include/oct.h"
#include "oct_internal.h"

namespace {

// Largest lattice side served: one 32-byte row record per lattice row.
constexpr int64_t kMaxRows = int64_t{1} << 17;
constexpr size_t kRowBytes = sizeof(oct::W2RowSums) * static_cast<size_t>(kMaxRows);
constexpr size_t kScratchBytes = kRowBytes + 256;  // rows, then the result block

static __device__ __align__(256) unsigned char g_w2_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
void *g_scratch_addr[kMaxDevices] = {};

// Device address of g_w2_scratch on the current device, looked up on the first
// call made with that device current.  The address belongs to the device's
// context at that call, so it does not survive a cudaDeviceReset of that
// device in the same process.
cudaError_t scratch_address(int dev, void **out) {
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_w2_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return cudaSuccess;
}

int fail(int code, const std::string &msg) {
    oct::set_last_error(msg);
    return code;
}

}  // namespace

extern "C" int oct_w2_noalloc(const void *lattice, int64_t L, void *stream, oct_w2 *out) {
    if (!lattice || !out) return fail(OCT_EINVAL, "oct_w2_noalloc: lattice and out must not be NULL");
    if (L < 64 || (L % 64) != 0)
        return fail(OCT_EINVAL, "oct_w2_noalloc: L must be a multiple of 64 and at least 64");
    if (L > kMaxRows)
        return fail(OCT_EINVAL, "oct_w2_noalloc: L = " + std::to_string(L) +
                                    " exceeds the largest lattice served without allocation (" +
                                    std::to_string(kMaxRows) + ")");
    if (reinterpret_cast<uintptr_t>(lattice) % 16u != 0u)
        return fail(OCT_EINVAL, "oct_w2_noalloc: the lattice must be 16-byte aligned");
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail(OCT_ECUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return fail(OCT_EUNSUPPORTED, "oct_w2_noalloc: device index too large");
    void *scratch = nullptr;
    e = scratch_address(dev, &scratch);
    if (e != cudaSuccess) return fail(OCT_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    auto *rows = static_cast<oct::W2RowSums *>(scratch);
    auto *res = reinterpret_cast<oct::W2Result *>(static_cast<unsigned char *>(scratch) + kRowBytes);
    // The kernels overwrite every row record and the whole result block before
    // they read them, so nothing left over from an earlier call needs clearing.
    e = oct::launch_w2(static_cast<const uint32_t *>(lattice), static_cast<uint32_t>(L), rows, res, st);
    oct::W2Result h;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h, res, sizeof(h), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return fail(OCT_ECUDA, std::string("oct_w2_noalloc: ") + cudaGetErrorString(e));
    const __int128 N = static_cast<__int128>(L) * L;
    const __int128 S2 = static_cast<__int128>((static_cast<unsigned __int128>(h.s2_hi) << 64) | h.s2_lo);
    const __int128 num = N * S2 - static_cast<__int128>(h.s1) * h.s1;
    out->t = -1;
    out->n_sites = static_cast<int64_t>(N);
    out->s1 = h.s1;
    out->s2_lo = h.s2_lo;
    out->s2_hi = h.s2_hi;
    out->net_flips = 0;
    out->hmax = h.hmax;
    out->w2 = static_cast<double>(num) / (static_cast<double>(N) * static_cast<double>(N));
    return OCT_OK;
}
