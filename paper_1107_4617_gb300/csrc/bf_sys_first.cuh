// Engine instantiations for the first (or only) harmonic chunk of a compact
// FP32 image on 128- or 64-thread strips: the seed is specialised at compile
// time (odd or even N) and every pair count 1..11 has its own kernel, with a
// half pair for an odd number of harmonics, so no harmonic is computed with a
// zero coefficient. Each translation unit bf_sys_first*.cu instantiates a few
// pair counts for one strip width (they compile in parallel). 64-thread strips
// (shared memory for 64 columns, four CTAs per SM) serve small images, whose
// 128-thread tiles would spend most steps in the skew ramp.
#pragma once
#include <type_traits>

#include "bf_sys_engine.cuh"

namespace bf {

// Form of the step per launch mode, seed (odd / even N), pair count and half
// pair. Bits 0-1, the step body: 0 = the four vertical streams one after
// another, then the centre; 1 = all five streams pair by pair; 2 / 3 = form
// 0 with the left neighbour's sums loaded two / one pair ahead of this
// lane's stores. Bit 2: the ping-pong step loop (two register sets for the
// pixels of consecutive steps, no copies between steps). Bit 3: the
// combine negates the box sums instead of the centre's sines. The forms
// compute the same values; they differ only in instruction schedule, and
// the fastest one differs between instantiations by up to 1.9x. Each entry
// was measured on a GB300 at 4096^2, r = 10 (median of 12 launches with L2
// flushed, every N = 2..43, all sixteen forms; a previous entry is kept
// unless another is at least 2 % faster), on 128-thread strips; the
// 64-thread kernels take the same forms.
constexpr unsigned char kFirstForm[3][2][11][2] = {
    // plain forward
    {
        {{14, 0}, {6, 5}, {6, 5}, {5, 5}, {11, 5}, {2, 4}, {0, 5}, {0, 5}, {0, 0}, {0, 0}, {0, 0}},
        {{5, 12}, {5, 6}, {6, 5}, {5, 5}, {5, 5}, {1, 5}, {0, 1}, {0, 0}, {1, 1}, {9, 0}, {0, 0}},
    },
    // forward with saved quads
    {
        {{13, 0}, {13, 13}, {5, 13}, {0, 5}, {0, 11}, {9, 12}, {8, 13}, {9, 0}, {9, 0}, {1, 9}, {8, 8}},
        {{13, 13}, {5, 12}, {4, 13}, {3, 8}, {2, 15}, {1, 0}, {8, 1}, {0, 0}, {0, 0}, {0, 8}, {0, 8}},
    },
    // adjoint
    {
        {{15, 0}, {6, 6}, {15, 13}, {15, 5}, {6, 13}, {1, 5}, {0, 6}, {8, 6}, {0, 0}, {8, 0}, {8, 8}},
        {{4, 6}, {6, 5}, {5, 6}, {15, 1}, {0, 5}, {0, 13}, {14, 13}, {8, 0}, {0, 0}, {8, 8}, {0, 1}},
    },
};

// Tin: the forward's input type. The adjoint reads only the saved quads, so it
// is instantiated for Tin = float alone.
template <int KP, bool HALF, int SEED, int WMAX, typename Tin>
cudaError_t sys_first_modes(const SysParams& p, int mode, int wi, int gx, int gy,
                            cudaStream_t s) {
    constexpr int F0 = kFirstForm[0][SEED - 1][KP - 1][HALF];
    constexpr int F1 = kFirstForm[1][SEED - 1][KP - 1][HALF];
    constexpr int F2 = kFirstForm[2][SEED - 1][KP - 1][HALF];
    // compact images only (p.ld == W): the pitch terms are compiled out
    if (mode == 2) {
        if constexpr (std::is_same<Tin, float>::value)
            return sys_launch_one<KP, true, false, false, WMAX, float, HALF, SEED, F2, false>(
                p, wi, gx, gy, s);
        else
            return cudaErrorInvalidValue;
    }
    if (mode == 1)
        return sys_launch_one<KP, false, true, false, WMAX, Tin, HALF, SEED, F1, false>(p, wi, gx,
                                                                                  gy, s);
    return sys_launch_one<KP, false, false, false, WMAX, Tin, HALF, SEED, F0, false>(p, wi, gx, gy,
                                                                                   s);
}

template <int KP, int WMAX, typename Tin>
cudaError_t sys_first_kp(const SysParams& p, int mode, bool half, int seed, int wi, int gx,
                         int gy, cudaStream_t s) {
    if (seed == 1)
        return half ? sys_first_modes<KP, true, 1, WMAX, Tin>(p, mode, wi, gx, gy, s)
                    : sys_first_modes<KP, false, 1, WMAX, Tin>(p, mode, wi, gx, gy, s);
    return half ? sys_first_modes<KP, true, 2, WMAX, Tin>(p, mode, wi, gx, gy, s)
                : sys_first_modes<KP, false, 2, WMAX, Tin>(p, mode, wi, gx, gy, s);
}

}  // namespace bf
