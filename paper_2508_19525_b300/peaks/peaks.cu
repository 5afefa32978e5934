// peaks.cu -- integer-pipe throughput of the arithmetic units the NTT and the
// base conversions are built from, for their ALU rooflines.  A measurement
// helper of the benchmark, built as its own library (libblb_peaks.so,
// include/blb_peaks.h); nothing on the hot path uses it.
//
// The NTT's unit of work is the lazy Cooley-Tukey butterfly on 64-bit words
// (one Shoup product by a constant twiddle, then X + WY and X - WY + 2q); the
// base conversions' unit is a 64 x 64 -> 128-bit multiply-accumulate, followed by
// one reduction of the 128-bit sum per output (blb_peaks_reduce_rate).  Each
// kernel runs independent chains of one unit entirely in registers (eight per
// thread, enough CTAs for every SM), so the measured rate is the integer
// pipes' throughput for that instruction mix with no memory traffic.  Every
// CTA also reports its SM cycles and nanoseconds, whose ratio is the SM clock
// during the run, so the rate is also known per SM cycle:
// peak = rate per SM cycle x SMs x SM clock.
#include <cuda_runtime.h>
#include <stdint.h>

#include "blb_peaks.h"

namespace {

struct acc128 {
    uint64_t lo, hi;
};
// acc += a b (mod 2^128), the multiply-add pair the base conversions use
__device__ __forceinline__ void mad128(acc128& acc, uint64_t a, uint64_t b)
{
    asm("mad.lo.cc.u64 %0, %2, %3, %0;\n\t"
        "madc.hi.u64 %1, %2, %3, %1;"
        : "+l"(acc.lo), "+l"(acc.hi)
        : "l"(a), "l"(b));
}

constexpr int PK_T = 256;
constexpr int PK_CHAINS = 8;

__device__ __forceinline__ uint64_t pk_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__global__ void __launch_bounds__(PK_T) k_peak_bfly(uint64_t* __restrict__ out, unsigned long long* __restrict__ cycles,
                                                    uint64_t w, uint64_t wp, uint64_t q, uint32_t iters)
{
    const uint64_t q2 = 2 * q;
    uint64_t x[PK_CHAINS], y[PK_CHAINS];
#pragma unroll
    for (int k = 0; k < PK_CHAINS; k++) {
        x[k] = (threadIdx.x * 7919ull + k * 104729ull + blockIdx.x) % q;
        y[k] = (threadIdx.x * 15485863ull + k * 32452843ull) % q;
    }
    const long long t0 = clock64();
    const uint64_t n0 = pk_ns();
    for (uint32_t it = 0; it < iters; it++) {
#pragma unroll
        for (int k = 0; k < PK_CHAINS; k++) {
            const uint64_t xr = x[k] >= q2 ? x[k] - q2 : x[k];
            const uint64_t t = y[k] * w - __umul64hi(y[k], wp) * q;
            x[k] = xr + t;
            y[k] = xr + q2 - t;
        }
    }
    const long long t1 = clock64();
    const uint64_t n1 = pk_ns();
    uint64_t r = 0;
#pragma unroll
    for (int k = 0; k < PK_CHAINS; k++) r ^= x[k] ^ y[k];
    out[blockIdx.x * PK_T + threadIdx.x] = r;
    if (threadIdx.x == 0) {
        atomicAdd(cycles, (unsigned long long)(t1 - t0));
        atomicAdd(cycles + 1, (unsigned long long)(n1 - n0));
    }
}

__global__ void __launch_bounds__(PK_T) k_peak_mad128(uint64_t* __restrict__ out,
                                                      unsigned long long* __restrict__ cycles, uint64_t h0,
                                                      uint64_t h1, uint32_t iters)
{
    uint64_t y[PK_CHAINS];
    acc128 a[PK_CHAINS];
#pragma unroll
    for (int k = 0; k < PK_CHAINS; k++) {
        y[k] = threadIdx.x * 2654435761ull + k * 40503ull + blockIdx.x;
        a[k] = acc128{0, 0};
    }
    const long long t0 = clock64();
    const uint64_t n0 = pk_ns();
    for (uint32_t it = 0; it < iters; it++) {
#pragma unroll
        for (int k = 0; k < PK_CHAINS; k++) {
            mad128(a[k], y[k], (it & 1) ? h1 : h0);
            y[k] += a[k].hi;
        }
    }
    const long long t1 = clock64();
    const uint64_t n1 = pk_ns();
    uint64_t r = 0;
#pragma unroll
    for (int k = 0; k < PK_CHAINS; k++) r ^= a[k].lo ^ a[k].hi;
    out[blockIdx.x * PK_T + threadIdx.x] = r;
    if (threadIdx.x == 0) {
        atomicAdd(cycles, (unsigned long long)(t1 - t0));
        atomicAdd(cycles + 1, (unsigned long long)(n1 - n0));
    }
}

// x mod q for a 128-bit x (the base conversions' and inner products' final
// reduction; the same three-product Barrett form as the library's)
__device__ __forceinline__ uint64_t barrett128(uint64_t x0, uint64_t x1, uint64_t q, uint64_t r0, uint64_t r1)
{
    const uint64_t qhat = x1 * r1 + __umul64hi(x1, r0) + __umul64hi(x0, r1);
    uint64_t r = x0 - qhat * q;
    const uint64_t q2 = q << 1;
    r = r >= q2 ? r - q2 : r;
    return r >= q ? r - q : r;
}

__global__ void __launch_bounds__(PK_T) k_peak_reduce(uint64_t* __restrict__ out,
                                                      unsigned long long* __restrict__ cycles, uint64_t q,
                                                      uint64_t r0, uint64_t r1, uint32_t iters)
{
    uint64_t x0[PK_CHAINS], x1[PK_CHAINS];
#pragma unroll
    for (int k = 0; k < PK_CHAINS; k++) {
        x0[k] = threadIdx.x * 2654435761ull + k * 40503ull + blockIdx.x;
        x1[k] = (threadIdx.x * 97ull + k) << 20;
    }
    const long long t0 = clock64();
    const uint64_t n0 = pk_ns();
    for (uint32_t it = 0; it < iters; it++) {
#pragma unroll
        for (int k = 0; k < PK_CHAINS; k++) {
            const uint64_t r = barrett128(x0[k], x1[k], q, r0, r1);
            x0[k] += r;  // the next input depends on this result
        }
    }
    const long long t1 = clock64();
    const uint64_t n1 = pk_ns();
    uint64_t r = 0;
#pragma unroll
    for (int k = 0; k < PK_CHAINS; k++) r ^= x0[k];
    out[blockIdx.x * PK_T + threadIdx.x] = r;
    if (threadIdx.x == 0) {
        atomicAdd(cycles, (unsigned long long)(t1 - t0));
        atomicAdd(cycles + 1, (unsigned long long)(n1 - n0));
    }
}

}  // namespace

extern "C" int blb_peaks_reduce_rate(uint64_t q, void* stream, double* per_s, double* per_sm_cycle)
{
    if (q < 3 || !(q & 1) || q >= (1ull << 62)) return -1;
    cudaStream_t st = (cudaStream_t)stream;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return -6;
    const uint32_t blocks = (uint32_t)sms * 8, iters = 4096;
    uint64_t* out = nullptr;
    unsigned long long* cyc = nullptr;
    if (cudaMalloc(&out, (size_t)blocks * PK_T * 8) != cudaSuccess) return -5;
    if (cudaMalloc(&cyc, 16) != cudaSuccess) {
        cudaFree(out);
        return -5;
    }
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const unsigned __int128 R = (~(unsigned __int128)0) / q;  // floor(2^128 / q) for odd q
    double rate = 0, per_cycle = 0;
    int rc = 0;
    for (int rep = 0; rep < 2 && !rc; rep++) {  // the first run warms up the clocks
        if (cudaMemsetAsync(cyc, 0, 16, st) != cudaSuccess) rc = -6;
        cudaEventRecord(e0, st);
        k_peak_reduce<<<blocks, PK_T, 0, st>>>(out, cyc, q, (uint64_t)R, (uint64_t)(R >> 64), iters);
        if (cudaGetLastError() != cudaSuccess) rc = -6;
        cudaEventRecord(e1, st);
        if (cudaEventSynchronize(e1) != cudaSuccess) rc = -6;
        float ms = 0;
        cudaEventElapsedTime(&ms, e0, e1);
        unsigned long long cn[2] = {0, 0};
        if (cudaMemcpy(cn, cyc, 16, cudaMemcpyDeviceToHost) != cudaSuccess) rc = -6;
        const double ops = (double)blocks * PK_T * iters * PK_CHAINS;
        const double ghz = cn[1] ? (double)cn[0] / (double)cn[1] : 1.0;
        rate = ops / (ms / 1e3);
        per_cycle = rate / ((double)sms * ghz * 1e9);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(out);
    cudaFree(cyc);
    if (rc) return rc;
    if (per_s) *per_s = rate;
    if (per_sm_cycle) *per_sm_cycle = per_cycle;
    return 0;
}

extern "C" int blb_peaks_int_rates(uint64_t q, void* stream, double* bfly_per_s, double* mad128_per_s,
                                   double* bfly_per_sm_cycle, double* mad128_per_sm_cycle)
{
    if (q < 3 || !(q & 1)) return -1;
    cudaStream_t st = (cudaStream_t)stream;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return -6;
    const uint32_t blocks = (uint32_t)sms * 8, iters = 4096;
    uint64_t* out = nullptr;
    unsigned long long* cyc = nullptr;
    if (cudaMalloc(&out, (size_t)blocks * PK_T * 8) != cudaSuccess) return -5;
    if (cudaMalloc(&cyc, 16) != cudaSuccess) {
        cudaFree(out);
        return -5;
    }
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    // a constant twiddle and its Shoup companion floor(w 2^64 / q)
    const uint64_t w = (q >> 3) + 12345, wp = (uint64_t)(((unsigned __int128)w << 64) / q);
    double res[2][2] = {{0, 0}, {0, 0}};
    int rc = 0;
    for (int kind = 0; kind < 2 && !rc; kind++) {
        for (int rep = 0; rep < 2 && !rc; rep++) {  // the first run warms up the clocks
            if (cudaMemsetAsync(cyc, 0, 16, st) != cudaSuccess) rc = -6;
            cudaEventRecord(e0, st);
            if (kind == 0)
                k_peak_bfly<<<blocks, PK_T, 0, st>>>(out, cyc, w, wp, q, iters);
            else
                k_peak_mad128<<<blocks, PK_T, 0, st>>>(out, cyc, w, wp, iters);
            if (cudaGetLastError() != cudaSuccess) rc = -6;
            cudaEventRecord(e1, st);
            if (cudaEventSynchronize(e1) != cudaSuccess) rc = -6;
            float ms = 0;
            cudaEventElapsedTime(&ms, e0, e1);
            unsigned long long cn[2] = {0, 0};
            if (cudaMemcpy(cn, cyc, 16, cudaMemcpyDeviceToHost) != cudaSuccess) rc = -6;
            const double ops = (double)blocks * PK_T * iters * PK_CHAINS;
            const double ghz = cn[1] ? (double)cn[0] / (double)cn[1] : 1.0;  // SM cycles per ns
            res[kind][0] = ops / (ms / 1e3);
            res[kind][1] = res[kind][0] / ((double)sms * ghz * 1e9);
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(out);
    cudaFree(cyc);
    if (rc) return rc;
    if (bfly_per_s) *bfly_per_s = res[0][0];
    if (bfly_per_sm_cycle) *bfly_per_sm_cycle = res[0][1];
    if (mad128_per_s) *mad128_per_s = res[1][0];
    if (mad128_per_sm_cycle) *mad128_per_sm_cycle = res[1][1];
    return 0;
}
