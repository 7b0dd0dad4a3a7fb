// Persistent batch kernel on the skewed-strip engine: each CTA pops tiles
// (image, strip, band) of one strip-width group from a device counter and runs
// every harmonic chunk of that tile in turn. Images are stored in decreasing
// order of per-tile cost, so the longest tiles start first. No CTA waits on
// another; the only device loop is over the finite tile list.
#include "bf_launch.cuh"
#include "bf_sys_engine.cuh"

namespace bf {

template <int KPMAX, int WMAX, typename Tin>
__device__ __forceinline__ void run_chunk(const SysParams& p, int kp, int bx, int by,
                                          float4* smem) {
    float gsum = 0.f;
    switch (kp) {
        case 1: sysd::sys_tile<1, false, false, false, WMAX, Tin>(p, bx, by, 0, 0, smem, gsum); break;
        case 2: sysd::sys_tile<2, false, false, false, WMAX, Tin>(p, bx, by, 0, 0, smem, gsum); break;
        case 3: sysd::sys_tile<3, false, false, false, WMAX, Tin>(p, bx, by, 0, 0, smem, gsum); break;
        case 4: sysd::sys_tile<4, false, false, false, WMAX, Tin>(p, bx, by, 0, 0, smem, gsum); break;
        case 6: sysd::sys_tile<6, false, false, false, WMAX, Tin>(p, bx, by, 0, 0, smem, gsum); break;
        case 8: sysd::sys_tile<8, false, false, false, WMAX, Tin>(p, bx, by, 0, 0, smem, gsum); break;
        default: sysd::sys_tile<KPMAX, false, false, false, WMAX, Tin>(p, bx, by, 0, 0, smem, gsum); break;
    }
}

template <int WMAX, typename Tin>
__global__ void __launch_bounds__(WMAX, 256 / WMAX) bf_sys_batch_kernel(SysBatchTable* tab,
                                                                        int group) {
    extern __shared__ float4 smem[];
    __shared__ SysParams sp;
    __shared__ int s_tile, s_img;
    if (tab->magic != SYS_BATCH_MAGIC) return;  // not a prepared table: no work
    const SysBatchGroup& G = tab->g[group];
    const int n_tiles = G.n_tiles;
    for (;;) {
        if (threadIdx.x == 0) {
            const int t = atomicAdd(&tab->counters[group], 1);
            s_tile = t;
            if (t < n_tiles) {
                // image holding tile t: last image whose first tile is <= t
                int lo = G.img0, hi = G.img0 + G.n_images - 1;
                while (lo < hi) {
                    const int mid = (lo + hi + 1) >> 1;
                    if (tab->img[mid].first_tile <= t) lo = mid; else hi = mid - 1;
                }
                s_img = lo;
            }
        }
        __syncthreads();
        const int t = s_tile;
        if (t >= n_tiles) break;
        const SysBatchImage& im = tab->img[s_img];
        const int local = t - im.first_tile;
        const int bx = local % im.gx, by = local / im.gx;
        for (int c = 0; c < im.nch; ++c) {
            __syncthreads();  // previous chunk / tile done with sp
            for (int i = threadIdx.x; i < (int)(sizeof(SysParams) / 4); i += blockDim.x)
                reinterpret_cast<int*>(&sp)[i] = reinterpret_cast<const int*>(&im.ch[c])[i];
            __syncthreads();
            run_chunk<SYS_KP_MAX, WMAX, Tin>(sp, im.kp[c], bx, by, smem);
        }
        __syncthreads();
    }
}

template <int WMAX, typename Tin>
static cudaError_t batch_launch(SysBatchTable* tab, int group, int wi, int grid, cudaStream_t s) {
    auto kern = bf_sys_batch_kernel<WMAX, Tin>;
    const size_t smem = sizeof(float4) * (size_t)sysd::sys_smem_slots(SYS_KP_MAX, WMAX);
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    kern<<<grid, wi, smem, s>>>(tab, group);
    return cudaGetLastError();
}

cudaError_t launch_sys_batch(SysBatchTable* tab, int group, int wi, int grid, int in_dtype,
                             cudaStream_t s) {
    if (wi <= 128) {
        return in_dtype == BF_BF16 ? batch_launch<128, __nv_bfloat16>(tab, group, wi, grid, s)
                                   : batch_launch<128, float>(tab, group, wi, grid, s);
    }
    return in_dtype == BF_BF16 ? batch_launch<256, __nv_bfloat16>(tab, group, wi, grid, s)
                               : batch_launch<256, float>(tab, group, wi, grid, s);
}

}  // namespace bf
