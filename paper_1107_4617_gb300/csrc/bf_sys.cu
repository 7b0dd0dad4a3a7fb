// Host dispatch of the skewed-strip engine (bf_sys_engine.cuh): picks the
// instantiation (strip width, harmonic pairs, seed, Kahan) and splits the harmonics
// of q_N's expansion into chunks when they exceed the register budget of one
// launch; chunks accumulate num/den (or the adjoint's two parts) in the
// output buffers and the last chunk finishes the ratio.
#include <string.h>

#include "bf_internal.cuh"

namespace bf {

// Harmonic-pair counts with their own instantiation; other counts run on the
// next larger one with zero coefficients for the extra harmonics.
static int sys_kp(int K) {
    static const int kps[] = {1, 2, 3, 4, 6, 8, 11};
    for (int kp : kps)
        if (2 * kp >= K) return kp;
    return -1;
}

// First-chunk kernels on 128- or 64-thread strips (wi <= 64 takes the
// 64-column instantiations; BF16 input of the forward has 128-thread ones;
// the adjoint reads only the saved quads and runs the FP32 ones): odd N
// (seed 1) runs kc harmonics in (kc + 1) / 2 pairs, even N (seed 2) the
// constant harmonic apart and kc - 1 harmonics in pairs; the last pair is
// half when the paired count is odd.
static cudaError_t launch_first(const SysParams& p, int mode, int kc, int seed, int wi, int gx,
                                int gy, bool bf16, cudaStream_t s) {
    const int np = seed == 2 ? kc - 1 : kc;
    const bool half = np & 1;
    if (wi <= 64) {
        switch ((np + 1) / 2) {
            case 1: return sys_first_kp<1, 64, float>(p, mode, half, seed, wi, gx, gy, s);
            case 2: return sys_first_kp<2, 64, float>(p, mode, half, seed, wi, gx, gy, s);
            case 3: return sys_first_kp<3, 64, float>(p, mode, half, seed, wi, gx, gy, s);
            case 4: return sys_first_kp<4, 64, float>(p, mode, half, seed, wi, gx, gy, s);
            case 5: return sys_first_kp<5, 64, float>(p, mode, half, seed, wi, gx, gy, s);
            case 6: return sys_first_kp<6, 64, float>(p, mode, half, seed, wi, gx, gy, s);
            case 7: return sys_first_kp<7, 64, float>(p, mode, half, seed, wi, gx, gy, s);
            case 8: return sys_first_kp<8, 64, float>(p, mode, half, seed, wi, gx, gy, s);
            case 9: return sys_first_kp<9, 64, float>(p, mode, half, seed, wi, gx, gy, s);
            case 10: return sys_first_kp<10, 64, float>(p, mode, half, seed, wi, gx, gy, s);
            case 11: return sys_first_kp<11, 64, float>(p, mode, half, seed, wi, gx, gy, s);
        }
        return cudaErrorInvalidValue;
    }
    if (bf16 && mode != 2) {
        switch ((np + 1) / 2) {
            case 1: return sys_first_kp<1, 128, __nv_bfloat16>(p, mode, half, seed, wi, gx, gy, s);
            case 2: return sys_first_kp<2, 128, __nv_bfloat16>(p, mode, half, seed, wi, gx, gy, s);
            case 3: return sys_first_kp<3, 128, __nv_bfloat16>(p, mode, half, seed, wi, gx, gy, s);
            case 4: return sys_first_kp<4, 128, __nv_bfloat16>(p, mode, half, seed, wi, gx, gy, s);
            case 5: return sys_first_kp<5, 128, __nv_bfloat16>(p, mode, half, seed, wi, gx, gy, s);
            case 6: return sys_first_kp<6, 128, __nv_bfloat16>(p, mode, half, seed, wi, gx, gy, s);
            case 7: return sys_first_kp<7, 128, __nv_bfloat16>(p, mode, half, seed, wi, gx, gy, s);
            case 8: return sys_first_kp<8, 128, __nv_bfloat16>(p, mode, half, seed, wi, gx, gy, s);
            case 9: return sys_first_kp<9, 128, __nv_bfloat16>(p, mode, half, seed, wi, gx, gy, s);
            case 10: return sys_first_kp<10, 128, __nv_bfloat16>(p, mode, half, seed, wi, gx, gy, s);
            case 11: return sys_first_kp<11, 128, __nv_bfloat16>(p, mode, half, seed, wi, gx, gy, s);
        }
        return cudaErrorInvalidValue;
    }
    switch ((np + 1) / 2) {
        case 1: return sys_first_kp<1, 128, float>(p, mode, half, seed, wi, gx, gy, s);
        case 2: return sys_first_kp<2, 128, float>(p, mode, half, seed, wi, gx, gy, s);
        case 3: return sys_first_kp<3, 128, float>(p, mode, half, seed, wi, gx, gy, s);
        case 4: return sys_first_kp<4, 128, float>(p, mode, half, seed, wi, gx, gy, s);
        case 5: return sys_first_kp<5, 128, float>(p, mode, half, seed, wi, gx, gy, s);
        case 6: return sys_first_kp<6, 128, float>(p, mode, half, seed, wi, gx, gy, s);
        case 7: return sys_first_kp<7, 128, float>(p, mode, half, seed, wi, gx, gy, s);
        case 8: return sys_first_kp<8, 128, float>(p, mode, half, seed, wi, gx, gy, s);
        case 9: return sys_first_kp<9, 128, float>(p, mode, half, seed, wi, gx, gy, s);
        case 10: return sys_first_kp<10, 128, float>(p, mode, half, seed, wi, gx, gy, s);
        case 11: return sys_first_kp<11, 128, float>(p, mode, half, seed, wi, gx, gy, s);
    }
    return cudaErrorInvalidValue;
}

int sys_chunks(int K, bool kahan, int kp_max) {
    int kp = kahan ? SYS_KP_KAHAN : SYS_KP_MAX;
    if (kp_max > 0 && kp_max < kp) kp = kp_max;
    const int per = 2 * kp;
    return (K + per - 1) / per;
}

cudaError_t launch_sys(const SysParams& base, int mode, bool kahan, int in_dtype, int wi, int gx,
                       int gy, cudaStream_t s, int kp_max) {
    if (wi > SYS_MAX_THREADS || wi % 32 != 0 || base.K < 1 || base.K > KCAP)
        return cudaErrorInvalidValue;
    if (kahan && mode == 2) return cudaErrorInvalidValue;
    const int nch = sys_chunks(base.K, kahan, kp_max);
    int per = (base.K + nch - 1) / nch;
    per += per & 1;  // whole harmonic pairs per chunk
    for (int c = 0; c < nch; ++c) {
        const int i0 = c * per;
        const int kc = (base.K - i0 < per) ? base.K - i0 : per;
        const int kp = kahan ? SYS_KP_KAHAN : sys_kp(kc);
        if (kp < 0) return cudaErrorInvalidValue;
        SysParams p = base;
        memset(p.a, 0, sizeof(p.a));
        memset(p.ak, 0, sizeof(p.ak));
        for (int i = 0; i < kc; ++i) {
            p.a[i] = base.a[i0 + i];
            p.ak[i] = base.a[i0 + i] * (float)(base.kstart + 2 * (i0 + i));
        }
        p.K = kc;
        p.k0 = base.kstart + 2 * i0;
        p.acc = (nch == 1) ? 0 : (c == 0 ? 1 : (c == nch - 1 ? 3 : 2));
        if (mode == 2 && c + 1 < nch) p.partial = nullptr;  // reduce only on the last chunk
        cudaError_t e;
        if (kahan) e = launch_sys_kahan(p, mode, in_dtype, kp, wi, gx, gy, s);
        else if (wi <= 128 && p.ld == p.W && (p.k0 == 1 || (p.k0 == 0 && kc > 1)) &&
                 (mode == 2 || in_dtype == BF_F32 || (in_dtype == BF_BF16 && wi > 64)))
            e = launch_first(p, mode, kc, p.k0 == 1 ? 1 : 2, wi, gx, gy,
                             mode != 2 && in_dtype == BF_BF16, s);
        else if (wi <= 128) e = launch_sys_w128(p, mode, in_dtype, kp, wi, gx, gy, s);
        else e = launch_sys_w256(p, mode, in_dtype, kp, wi, gx, gy, s);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace bf
