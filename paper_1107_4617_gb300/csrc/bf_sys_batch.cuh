// Persistent batch kernels on the skewed-strip engine: each CTA pops tiles
// (image, strip, band) of one group from a device counter and runs every
// harmonic chunk of that tile in turn. Images are stored in decreasing order
// of per-tile cost, so the longest tiles start first. No CTA waits on
// another; the only device loop is over the finite tile list.
//
// Groups (SysBatchTable::g), one persistent launch each:
//  0: 128-thread images whose harmonics fit one chunk of at most
//     SYS_BATCH_SMALL_KP pairs (small N: most images of a batch whose sigma_r
//     spreads over [0.08, 0.4]); the kernel switches between the first-chunk
//     specialisations (compile-time seed, half pair, the measured step
//     form), whose registers allow three CTAs per SM;
//  1: the other 128-thread images, the general kernel (two CTAs per SM);
//  2: 256-thread strips (r > 40), the general kernel.
// Template SPEC: 0 general, 1 group 0. (The same specialisations for group 1,
// one chunk of 5..11 pairs, measured slower than the general kernel there:
// 23.1 against 24.7 Gpx/s on the 256-image batch; a separate launch for its
// two-chunk images, slower still, 21.5.)
#pragma once
#include "bf_launch.cuh"
#include "bf_sys_first.cuh"

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

// One tile of a group-0 image: the plain-forward specialisation for (KP,
// HALF, SEED) with its measured step form; row pitch kept.
template <int KP, bool HALF, int SEED, typename Tin>
__device__ __forceinline__ void small_tile(const SysParams& p, int bx, int by, float4* smem) {
    constexpr int F = kFirstForm[0][SEED - 1][KP - 1][HALF];
    float gsum = 0.f;
    sysd::sys_tile<KP, false, false, false, 128, Tin, HALF, SEED, F, true>(p, bx, by, 0, 0, smem,
                                                                          gsum);
}

template <typename Tin>
__device__ __forceinline__ void run_small(const SysParams& p, int kind, int bx, int by,
                                          float4* smem) {
    switch (kind) {
        case 0: small_tile<1, false, 1, Tin>(p, bx, by, smem); break;
        case 1: small_tile<1, true, 1, Tin>(p, bx, by, smem); break;
        case 2: small_tile<2, false, 1, Tin>(p, bx, by, smem); break;
        case 3: small_tile<2, true, 1, Tin>(p, bx, by, smem); break;
        case 4: small_tile<3, false, 1, Tin>(p, bx, by, smem); break;
        case 5: small_tile<3, true, 1, Tin>(p, bx, by, smem); break;
        case 6: small_tile<4, false, 1, Tin>(p, bx, by, smem); break;
        case 7: small_tile<4, true, 1, Tin>(p, bx, by, smem); break;
        case 8: small_tile<1, false, 2, Tin>(p, bx, by, smem); break;
        case 9: small_tile<1, true, 2, Tin>(p, bx, by, smem); break;
        case 10: small_tile<2, false, 2, Tin>(p, bx, by, smem); break;
        case 11: small_tile<2, true, 2, Tin>(p, bx, by, smem); break;
        case 12: small_tile<3, false, 2, Tin>(p, bx, by, smem); break;
        case 13: small_tile<3, true, 2, Tin>(p, bx, by, smem); break;
        case 14: small_tile<4, false, 2, Tin>(p, bx, by, smem); break;
        default: small_tile<4, true, 2, Tin>(p, bx, by, smem); break;
    }
}

constexpr int SMALL_CTAS_PER_SM = 3;

template <int WMAX, typename Tin, int SPEC>
__global__ void __launch_bounds__(WMAX, SPEC == 1 ? SMALL_CTAS_PER_SM : 256 / WMAX)
    bf_sys_batch_kernel(SysBatchTable* tab, int group) {
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
            if constexpr (SPEC == 1) run_small<Tin>(sp, im.kind, bx, by, smem);
            else run_chunk<SYS_KP_MAX, WMAX, Tin>(sp, im.kp[c], bx, by, smem);
        }
        __syncthreads();
    }
}

template <int WMAX, typename Tin, int SPEC>
static size_t batch_smem() {
    return sizeof(float4) *
           (size_t)(SPEC == 1 ? sysd::sys_smem_slots(SYS_BATCH_SMALL_KP, WMAX, true)
                              : sysd::sys_smem_slots(SYS_KP_MAX, WMAX));
}

template <int WMAX, typename Tin, int SPEC>
cudaError_t batch_launch(SysBatchTable* tab, int group, int grid, cudaStream_t s) {
    auto kern = bf_sys_batch_kernel<WMAX, Tin, SPEC>;
    const size_t smem = batch_smem<WMAX, Tin, SPEC>();
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    kern<<<grid, WMAX, smem, s>>>(tab, group);
    return cudaGetLastError();
}

template <int WMAX, typename Tin, int SPEC>
int batch_grid() {
    auto kern = bf_sys_batch_kernel<WMAX, Tin, SPEC>;
    const size_t smem = batch_smem<WMAX, Tin, SPEC>();
    int per_sm = 0;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
            cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, WMAX, smem) != cudaSuccess ||
        per_sm < 1)
        per_sm = 1;
    return per_sm * sm_count();
}

}  // namespace bf
