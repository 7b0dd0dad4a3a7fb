// bf_check_range: min and max of an image, so a caller can check the filter's
// precondition that all values lie in an interval of length T (Sec. 3: the
// range kernel is a valid kernel on [-T, T] only). Also the variants' band
// height rule.
#include <math.h>

#include "bf_internal.cuh"
#include "bf_quads.cuh"
#include "bf_launch.cuh"
#include "bf_trace.cuh"

namespace bf {
namespace util {

// Order-preserving map of float bits to int (and back): x < y as floats iff
// key(x) < key(y) as ints, for every non-NaN value.
__device__ __forceinline__ int fkey(float x) {
    const int b = __float_as_int(x);
    return b >= 0 ? b : b ^ 0x7fffffff;
}
__device__ __forceinline__ float fkey_inv(int k) {
    return __int_as_float(k >= 0 ? k : k ^ 0x7fffffff);
}

__global__ void init_kernel(int* keys) {
    keys[0] = 0x7fffffff;            // key of +max: min starts above everything
    keys[1] = (int)0x80000000;       // max starts below everything
}

template <typename T>
__device__ __forceinline__ float load_val(const T* p, size_t i);
template <>
__device__ __forceinline__ float load_val<float>(const float* p, size_t i) { return __ldg(p + i); }
template <>
__device__ __forceinline__ float load_val<__nv_bfloat16>(const __nv_bfloat16* p, size_t i) {
    return __bfloat162float(p[i]);
}

template <typename T>
__global__ void minmax_kernel(const T* img, size_t n, int* keys) {
    int kmin = 0x7fffffff, kmax = (int)0x80000000;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
         i += (size_t)gridDim.x * blockDim.x) {
        const int k = fkey(load_val<T>(img, i));
        kmin = min(kmin, k);
        kmax = max(kmax, k);
    }
    for (int o = 16; o > 0; o >>= 1) {
        kmin = min(kmin, __shfl_down_sync(0xffffffffu, kmin, o));
        kmax = max(kmax, __shfl_down_sync(0xffffffffu, kmax, o));
    }
    __shared__ int smin[32], smax[32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) { smin[w] = kmin; smax[w] = kmax; }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int q = 1; q < (int)(blockDim.x >> 5); ++q) {
            kmin = min(kmin, smin[q]);
            kmax = max(kmax, smax[q]);
        }
        atomicMin(keys, kmin);
        atomicMax(keys + 1, kmax);
    }
}

__global__ void finish_kernel(int* keys) {
    float* f = reinterpret_cast<float*>(keys);
    const float lo = fkey_inv(keys[0]), hi = fkey_inv(keys[1]);
    f[0] = lo;
    f[1] = hi;
}

}  // namespace util

// out = f and the quads (f, 1, f, 0), pixel (y, x)'s at quad_index64(y, x, H, W)
__global__ void unit_window_quads(const float* img, float* out, float4* sv, int H, int W) {
    const size_t n = (size_t)H * W;
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += stride) {
        const float f = img[i];
        const int y = (int)(i / (size_t)W), x = (int)(i - (size_t)y * W);
        out[i] = f;
        sv[quad_index64(y, x, H, W)] = make_float4(f, 1.f, f, 0.f);
    }
}

cudaError_t unit_window(const float* img, float* out, float4* sv, int H, int W, cudaStream_t s) {
    const size_t n = (size_t)H * W;
    if (!sv) return cudaMemcpyAsync(out, img, sizeof(float) * n, cudaMemcpyDeviceToDevice, s);
    const size_t want = (n + 255) / 256, cap = (size_t)8 * sm_count();
    unit_window_quads<<<(unsigned)(want < cap ? want : cap), 256, 0, s>>>(img, out, sv, H, W);
    return cudaGetLastError();
}

int wave_band_rows(const void* kern, int threads, size_t smem, int H, int gx) {
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, threads, smem) != cudaSuccess ||
        occ < 1)
        occ = 1;
    int nb = occ * sm_count() / (gx > 0 ? gx : 1);  // rounding up would start a second wave
    if (nb < 1) nb = 1;
    int hb = (H + nb - 1) / nb;
    return hb < 32 ? 32 : hb;
}

}  // namespace bf

using namespace bf;

extern "C" size_t bf_saved_index(int y, int x, int H, int W) {
    if (H < 1 || W < 1 || y < 0 || y >= H || x < 0 || x >= W) return (size_t)-1;
    return quad_index64(y, x, H, W);
}

extern "C" bf_status bf_check_range(const void* img, int H, int W, int in_dtype, float* minmax,
                                    void* stream) {
    BF_TRACE("bf_check_range");
    if (!img || !minmax || H < 1 || W < 1) return BF_ERR_INVALID_ARG;
    if (in_dtype != BF_F32 && in_dtype != BF_BF16) return BF_ERR_INVALID_ARG;
    if ((uintptr_t)minmax & 7) return BF_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    int* keys = reinterpret_cast<int*>(minmax);
    const size_t n = (size_t)H * W;
    int grid = 2 * sm_count();
    if ((size_t)grid * 256 > n) grid = (int)((n + 255) / 256);
    util::init_kernel<<<1, 1, 0, s>>>(keys);
    if (in_dtype == BF_BF16)
        util::minmax_kernel<__nv_bfloat16>
            <<<grid, 256, 0, s>>>(static_cast<const __nv_bfloat16*>(img), n, keys);
    else
        util::minmax_kernel<float><<<grid, 256, 0, s>>>(static_cast<const float*>(img), n, keys);
    util::finish_kernel<<<1, 1, 0, s>>>(keys);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return set_cuda_error(e);
    return BF_OK;
}
