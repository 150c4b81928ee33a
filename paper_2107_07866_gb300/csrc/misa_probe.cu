// misa_probe.cu -- issue-rate microbenchmarks of the pipes the EAM gathers
// and the FP64 integration use: scalar FP32 FMA, packed FP32x2 FMA, FP64 FMA,
// the MUFU reciprocal square root, and conflict-free 16-byte shared-memory
// loads.  They give the denominators of the "alu" roofline measured on the
// device itself rather than derived from unit counts and the clock.
//
// Every kernel runs a fixed number of iterations of independent dependency
// chains (enough chains per warp to hide the pipe latency), grid-filled with
// several CTAs per SM; the result is stored only when it equals an
// impossible value, so the compiler keeps the work.  Device time from CUDA
// events on the caller's stream; the SM clock during the probe from
// clock64() against %globaltimer in the first CTA of the FP32 probe.  Nothing here changes a
// device setting.
#include <cuda_runtime.h>

#include <cstdint>

#include "misa.h"

namespace {

constexpr int kThreads = 512;
constexpr int kChains = 8;

__device__ float g_sink_f;
__device__ double g_sink_d;
__device__ unsigned g_sink_u;
__device__ unsigned long long g_clock[4];

__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__global__ void __launch_bounds__(kThreads) k_ffma(int iters, float b, float c)
{
    const bool timer = blockIdx.x == 0 && threadIdx.x == 0;
    unsigned long long c0 = 0, t0 = 0;
    if (timer) {
        c0 = clock64();
        t0 = global_ns();
    }
    float a[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = (float)(threadIdx.x + k);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int r = 0; r < 16; ++r)
#pragma unroll
            for (int k = 0; k < kChains; ++k) a[k] = fmaf(a[k], b, c);
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += a[k];
    if (s == -1.2345f) g_sink_f = s;
    if (timer) {  // SM cycles and nanoseconds of the first CTA under full load
        g_clock[0] = clock64() - c0;
        g_clock[1] = global_ns() - t0;
    }
}

__global__ void __launch_bounds__(kThreads) k_ffma2(int iters, float b, float c)
{
    float2 a[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = make_float2((float)(threadIdx.x + k), (float)(k - (int)threadIdx.x));
    const float2 b2 = make_float2(b, b), c2 = make_float2(c, c);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int r = 0; r < 16; ++r)
#pragma unroll
            for (int k = 0; k < kChains; ++k) a[k] = __ffma2_rn(a[k], b2, c2);
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += a[k].x + a[k].y;
    if (s == -1.2345f) g_sink_f = s;
}

__global__ void __launch_bounds__(kThreads) k_dfma(int iters, double b, double c)
{
    double a[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = (double)(threadIdx.x + k);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int r = 0; r < 16; ++r)
#pragma unroll
            for (int k = 0; k < kChains; ++k) a[k] = fma(a[k], b, c);
    }
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += a[k];
    if (s == -1.2345) g_sink_d = s;
}

__global__ void __launch_bounds__(kThreads) k_mufu(int iters)
{
    float a[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = 1.0f + (float)(threadIdx.x + k);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int r = 0; r < 16; ++r)
#pragma unroll
            for (int k = 0; k < kChains; ++k) asm volatile("rsqrt.approx.ftz.f32 %0, %0;" : "+f"(a[k]));
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += a[k];
    if (s == -1.2345f) g_sink_f = s;
}

// 16-byte loads: the 32 lanes of a warp read 32 consecutive 16-byte words
// (eight lanes cover all 32 banks once per quarter warp: conflict-free, four
// wavefronts a warp), at addresses that move every iteration so that no
// load can be hoisted or merged
constexpr int kLdsWords = 2048;
__global__ void __launch_bounds__(kThreads) k_lds(int iters)
{
    __shared__ uint4 buf[kLdsWords];
    for (int q = threadIdx.x; q < kLdsWords; q += kThreads) buf[q] = make_uint4(q, q * 3u, q * 5u, q * 7u);
    __syncthreads();
    uint4 acc = make_uint4(0, 0, 0, 0);
    const unsigned lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
    const unsigned base = (unsigned)__cvta_generic_to_shared(buf);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int k = 0; k < kChains; ++k) {
            const unsigned word = (lane + 32u * (warp + (unsigned)(kChains * it + k))) & (kLdsWords - 1);
            uint4 v;
            asm volatile("ld.shared.v4.u32 {%0, %1, %2, %3}, [%4];"
                         : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
                         : "r"(base + 16u * word));
            acc.x += v.x;
            acc.y ^= v.y;
            acc.z += v.z;
            acc.w ^= v.w;
        }
    }
    if ((acc.x ^ acc.y ^ acc.z ^ acc.w) == 0x9e3779b9u) g_sink_u = acc.x;
}

struct Timer {
    cudaEvent_t a = nullptr, b = nullptr;
    cudaStream_t st;
    explicit Timer(cudaStream_t s) : st(s)
    {
        cudaEventCreate(&a);
        cudaEventCreate(&b);
    }
    ~Timer()
    {
        if (a) cudaEventDestroy(a);
        if (b) cudaEventDestroy(b);
    }
};

// best of `reps` timed launches (ms) of launch(); one untimed launch first
template <typename F>
cudaError_t best_ms(Timer &t, int reps, F launch, double &ms)
{
    launch();
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    ms = 1e30;
    for (int r = 0; r < reps; ++r) {
        cudaEventRecord(t.a, t.st);
        launch();
        cudaEventRecord(t.b, t.st);
        e = cudaEventSynchronize(t.b);
        if (e != cudaSuccess) return e;
        float x = 0.f;
        cudaEventElapsedTime(&x, t.a, t.b);
        if (x < ms) ms = x;
    }
    return cudaGetLastError();
}

}  // namespace

extern "C" int misa_measure_peaks(misa_peaks *out, void *stream)
{
    if (!out) return MISA_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    int dev = 0, nsm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return MISA_ECUDA;
    if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || nsm <= 0) return MISA_ECUDA;
    Timer t(st);
    if (!t.a || !t.b) return MISA_ECUDA;
    const int grid = 4 * nsm;  // 4 CTAs of 512 threads: every warp slot of an SM
    const double threads = (double)grid * kThreads;
    const int reps = 5;
    double ms = 0.0;
    cudaError_t e;

    const int it_f = 8192;  // 16 x 8 FMAs per iteration per thread
    e = best_ms(t, reps, [&] { k_ffma<<<grid, kThreads, 0, st>>>(it_f, 0.9999f, 1e-6f); }, ms);
    if (e != cudaSuccess) return MISA_ECUDA;
    out->fp32_ffma_tflops = 2.0 * 16 * kChains * (double)it_f * threads / (ms * 1e-3) / 1e12;

    e = best_ms(t, reps, [&] { k_ffma2<<<grid, kThreads, 0, st>>>(it_f / 2, 0.9999f, 1e-6f); }, ms);
    if (e != cudaSuccess) return MISA_ECUDA;
    out->fp32_ffma2_tflops = 4.0 * 16 * kChains * (double)(it_f / 2) * threads / (ms * 1e-3) / 1e12;

    const int it_d = 64;
    e = best_ms(t, reps, [&] { k_dfma<<<grid, kThreads, 0, st>>>(it_d, 0.9999, 1e-6); }, ms);
    if (e != cudaSuccess) return MISA_ECUDA;
    out->fp64_dfma_tflops = 2.0 * 16 * kChains * (double)it_d * threads / (ms * 1e-3) / 1e12;

    const int it_m = 512;
    e = best_ms(t, reps, [&] { k_mufu<<<grid, kThreads, 0, st>>>(it_m); }, ms);
    if (e != cudaSuccess) return MISA_ECUDA;
    out->mufu_rsqrt_tops = 16.0 * kChains * (double)it_m * threads / (ms * 1e-3) / 1e12;

    const int it_l = 4096;
    e = best_ms(t, reps, [&] { k_lds<<<grid, kThreads, 0, st>>>(it_l); }, ms);
    if (e != cudaSuccess) return MISA_ECUDA;
    out->lds128_tbps = 16.0 * kChains * (double)it_l * threads / (ms * 1e-3) / 1e12;

    unsigned long long h[2] = {0, 0};
    if (cudaMemcpyFromSymbol(h, g_clock, sizeof(h)) != cudaSuccess) return MISA_ECUDA;
    out->sm_clock_mhz = h[1] ? 1e3 * (double)h[0] / (double)h[1] : 0.0;
    out->num_sms = nsm;
    return MISA_OK;
}
