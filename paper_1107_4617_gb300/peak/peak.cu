// Throughput micro-benchmarks of the pipes the filter's kernels use: FP32 FMA
// (scalar and packed FP32x2), FP32 add, warp shuffle, 128-bit shared loads and
// the MUFU sine. Each kernel runs 8 independent dependency chains per thread
// over 8 CTAs per SM, long enough to dominate launch overhead; the result is
// printed as one JSON object (rates at the measured duration, not at a fixed
// clock).
#include <cstdio>
#include <cuda_runtime.h>

#define CHK(x) do { cudaError_t e = (x); if (e != cudaSuccess) { printf("CUDA %s line %d\n", cudaGetErrorString(e), __LINE__); return 1; } } while (0)

constexpr int ITERS = 4096;

__global__ void k_ffma(float* out, float a, float b) {
    float x[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) x[i] = threadIdx.x * 0.001f + i;
    for (int it = 0; it < ITERS; ++it) {
#pragma unroll
        for (int i = 0; i < 8; ++i) x[i] = fmaf(x[i], a, b);
    }
    float s = 0; for (int i = 0; i < 8; ++i) s += x[i];
    if (s == 1.2345f) out[0] = s;
}

__global__ void k_ffma2(float* out, float a, float b) {
    float2 x[8];
    const float2 A = make_float2(a, a), B = make_float2(b, b);
#pragma unroll
    for (int i = 0; i < 8; ++i) x[i] = make_float2(threadIdx.x * 0.001f + i, i * 0.5f);
    for (int it = 0; it < ITERS; ++it) {
#pragma unroll
        for (int i = 0; i < 8; ++i) x[i] = __ffma2_rn(x[i], A, B);
    }
    float s = 0; for (int i = 0; i < 8; ++i) s += x[i].x + x[i].y;
    if (s == 1.2345f) out[0] = s;
}

__global__ void k_fadd2(float* out, float a) {
    float2 x[8];
    const float2 A = make_float2(a, -a);
#pragma unroll
    for (int i = 0; i < 8; ++i) x[i] = make_float2(threadIdx.x * 0.001f + i, i * 0.5f);
    for (int it = 0; it < ITERS; ++it) {
#pragma unroll
        for (int i = 0; i < 8; ++i) x[i] = __fadd2_rn(x[i], A);
    }
    float s = 0; for (int i = 0; i < 8; ++i) s += x[i].x + x[i].y;
    if (s == 1.2345f) out[0] = s;
}

__global__ void k_fadd(float* out, float a) {
    float x[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) x[i] = threadIdx.x * 0.001f + i;
    for (int it = 0; it < ITERS; ++it) {
#pragma unroll
        for (int i = 0; i < 8; ++i) x[i] = x[i] + a;
    }
    float s = 0; for (int i = 0; i < 8; ++i) s += x[i];
    if (s == 1.2345f) out[0] = s;
}

__global__ void k_shfl(float* out) {
    float x[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) x[i] = threadIdx.x * 0.001f + i;
    for (int it = 0; it < ITERS / 4; ++it) {
#pragma unroll
        for (int i = 0; i < 4; ++i) x[i] = __shfl_up_sync(0xffffffffu, x[i], 1);
    }
    float s = 0; for (int i = 0; i < 4; ++i) s += x[i];
    if (s == 1.2345f) out[0] = s;
}

__global__ void k_lds(float* out) {
    __shared__ float4 buf[1024];
    for (int i = threadIdx.x; i < 1024; i += blockDim.x) buf[i] = make_float4(i, i, i, i);
    __syncthreads();
    float4 acc = make_float4(0, 0, 0, 0);
    int idx = threadIdx.x;
    for (int it = 0; it < ITERS / 4; ++it) {
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            float4 v = buf[(idx + i * 32) & 1023];
            acc.x += v.x; acc.y += v.y; acc.z += v.z; acc.w += v.w;
        }
        idx += 7;
    }
    if (acc.x == 1.2345f) out[0] = acc.x + acc.y + acc.z + acc.w;
}

__global__ void k_mufu(float* out, float a) {
    float x[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) x[i] = threadIdx.x * 0.001f + i;
    for (int it = 0; it < ITERS / 4; ++it) {
#pragma unroll
        for (int i = 0; i < 8; ++i) x[i] = __sinf(x[i]) + a;
    }
    float s = 0; for (int i = 0; i < 8; ++i) s += x[i];
    if (s == 1.2345f) out[0] = s;
}

int main() {
    int dev = 0, sms = 0, clk = 0;
    CHK(cudaGetDevice(&dev));
    CHK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    CHK(cudaDeviceGetAttribute(&clk, cudaDevAttrClockRate, dev));
    printf("{\"sms\": %d, \"max_clock_khz\": %d", sms, clk);
    float* out; CHK(cudaMalloc(&out, 16));
    cudaEvent_t e0, e1; cudaEventCreate(&e0); cudaEventCreate(&e1);
    const int blocks = sms * 8, threads = 256;
    const double nthreads = (double)blocks * threads;
    auto timeit = [&](auto launch) -> double {
        for (int w = 0; w < 3; ++w) launch();
        cudaEventRecord(e0);
        for (int w = 0; w < 5; ++w) launch();
        cudaEventRecord(e1);
        cudaEventSynchronize(e1);
        float ms; cudaEventElapsedTime(&ms, e0, e1);
        return ms / 5 / 1e3;
    };
    double t;
    t = timeit([&] { k_ffma<<<blocks, threads>>>(out, 0.999f, 0.001f); });
    printf(", \"ffma_tflops\": %.2f", nthreads * ITERS * 8 * 2 / t / 1e12);
    t = timeit([&] { k_ffma2<<<blocks, threads>>>(out, 0.999f, 0.001f); });
    printf(", \"ffma2_tflops\": %.2f", nthreads * ITERS * 8 * 4 / t / 1e12);
    t = timeit([&] { k_fadd<<<blocks, threads>>>(out, 0.001f); });
    printf(", \"fadd_tops\": %.2f", nthreads * ITERS * 8 / t / 1e12);
    t = timeit([&] { k_fadd2<<<blocks, threads>>>(out, 0.001f); });
    printf(", \"fadd2_tops\": %.2f", nthreads * ITERS * 8 * 2 / t / 1e12);
    t = timeit([&] { k_shfl<<<blocks, threads>>>(out); });
    printf(", \"shfl_lanes_per_clk_sm\": %.2f", nthreads * ITERS / t / (clk * 1e3) / sms);
    t = timeit([&] { k_lds<<<blocks, threads>>>(out); });
    printf(", \"lds128_bytes_per_clk_sm\": %.1f", nthreads * ITERS * 16 / t / (clk * 1e3) / sms);
    t = timeit([&] { k_mufu<<<blocks, threads>>>(out, 0.1f); });
    printf(", \"mufu_sin_lanes_per_clk_sm\": %.2f}\n", nthreads * ITERS * 2 / t / (clk * 1e3) / sms);
    return 0;
}
