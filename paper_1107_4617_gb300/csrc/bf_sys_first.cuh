// Engine instantiations for the first (or only) harmonic chunk of an FP32
// image on 128-thread strips: the seed is specialised at compile time (odd or
// even N) and every pair count 1..11 has its own kernel, with a half pair for
// an odd number of harmonics, so no harmonic is computed with a zero
// coefficient. Each translation unit bf_sys_first*.cu instantiates a few
// pair counts (they compile in parallel).
#pragma once
#include "bf_sys_engine.cuh"

namespace bf {

template <int KP, bool HALF, int SEED>
cudaError_t sys_first_modes(const SysParams& p, int mode, int wi, int gx, int gy,
                            cudaStream_t s) {
    if (mode == 2)
        return sys_launch_one<KP, true, false, false, 128, float, HALF, SEED>(p, wi, gx, gy, s);
    if (mode == 1)
        return sys_launch_one<KP, false, true, false, 128, float, HALF, SEED>(p, wi, gx, gy, s);
    return sys_launch_one<KP, false, false, false, 128, float, HALF, SEED>(p, wi, gx, gy, s);
}

template <int KP>
cudaError_t sys_first_kp(const SysParams& p, int mode, bool half, int seed, int wi, int gx,
                         int gy, cudaStream_t s) {
    if (seed == 1)
        return half ? sys_first_modes<KP, true, 1>(p, mode, wi, gx, gy, s)
                    : sys_first_modes<KP, false, 1>(p, mode, wi, gx, gy, s);
    return half ? sys_first_modes<KP, true, 2>(p, mode, wi, gx, gy, s)
                : sys_first_modes<KP, false, 2>(p, mode, wi, gx, gy, s);
}

}  // namespace bf
