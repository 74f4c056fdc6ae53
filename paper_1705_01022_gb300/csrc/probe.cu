// Integer-pipe throughput probe: the denominator of the hot path's roofline.
//
// The device-step kernel is bound by 32-bit integer logic (LOP3, shifts,
// IMAD for the Philox multiplications).  This probe runs long chains of
// independent LOP3 (three-input logic) or IMAD (32-bit multiply-add)
// instructions on every SM, reads the SM cycle counter around the chains, and
// returns operations per SM per clock together with the clock the SMs ran at.
#include <cuda_runtime.h>

#include "oct_internal.h"

namespace oct {
namespace {

constexpr int kChains = 8;
constexpr int kIters = 4096;

template <int OP>
__global__ void __launch_bounds__(1024) int_rate_kernel(uint32_t seed, uint32_t *sink,
                                                         unsigned long long *cycles) {
    uint32_t a[kChains];
#pragma unroll
    for (int i = 0; i < kChains; ++i) a[i] = seed ^ (threadIdx.x * 0x9E3779B9u + i);
    const uint32_t b = seed * 3u + blockIdx.x, c = seed ^ 0x5bd1e995u;
    __syncthreads();
    const long long c0 = clock64();
    for (int it = 0; it < kIters; ++it) {
#pragma unroll
        for (int i = 0; i < kChains; ++i) {
            if (OP == 0)
                asm volatile("lop3.b32 %0, %0, %1, %2, 0x96;" : "+r"(a[i]) : "r"(b), "r"(c));
            else
                asm volatile("mad.lo.u32 %0, %0, %1, %2;" : "+r"(a[i]) : "r"(b), "r"(c));
        }
    }
    __syncthreads();
    const long long c1 = clock64();
    uint32_t x = 0;
#pragma unroll
    for (int i = 0; i < kChains; ++i) x ^= a[i];
    if (x == 0x12345678u) sink[0] = x;  // keeps the chains live
    if (threadIdx.x == 0) atomicMax(cycles, static_cast<unsigned long long>(c1 - c0));
}

}  // namespace

cudaError_t measure_int_rate(int op, int sms, double *ops_per_clk_per_sm, double *mhz) {
    uint32_t *sink = nullptr;
    unsigned long long *cyc = nullptr;
    cudaError_t e = cudaMalloc(&sink, 4);
    if (e == cudaSuccess) e = cudaMalloc(&cyc, 8);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    const int blocks = 2 * sms, threads = 1024;
    float ms = 0.f;
    unsigned long long c = 0;
    for (int rep = 0; rep < 2 && e == cudaSuccess; ++rep) {  // first pass warms up
        e = cudaMemset(cyc, 0, 8);
        if (e == cudaSuccess) e = cudaEventRecord(e0);
        if (e == cudaSuccess) {
            if (op == 0)
                int_rate_kernel<0><<<blocks, threads>>>(1u, sink, cyc);
            else
                int_rate_kernel<1><<<blocks, threads>>>(1u, sink, cyc);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) e = cudaEventRecord(e1);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e == cudaSuccess) e = cudaMemcpy(&c, cyc, 8, cudaMemcpyDeviceToHost);
    }
    if (e == cudaSuccess) {
        // each SM runs two blocks back to back at most; total ops / (SMs * cycles of the
        // longest block * blocks per SM in sequence) is conservative, so use the event time.
        const double ops = static_cast<double>(blocks) * threads * kIters * kChains;
        const double clk_hz = static_cast<double>(c) / (ms * 1e-3 / 1.0);
        // c is the cycles of one block's chain; blocks are resident together when two fit
        // per SM, so the wall time covers about c cycles.
        *mhz = clk_hz * 1e-6;
        *ops_per_clk_per_sm = ops / (static_cast<double>(sms) * static_cast<double>(c));
    }
    if (sink) cudaFree(sink);
    if (cyc) cudaFree(cyc);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    return e;
}

}  // namespace oct
