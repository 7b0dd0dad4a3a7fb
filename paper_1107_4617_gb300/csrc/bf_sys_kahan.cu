// Instantiations of the skewed-strip engine with Kahan-compensated vertical
// running sums (forward only; 6 harmonic pairs per chunk so the compensation
// registers fit beside the sums).
#include "bf_sys_engine.cuh"

namespace bf {

cudaError_t launch_sys_kahan(const SysParams& p, int mode, int dtype, int kp, int wi, int gx,
                             int gy, cudaStream_t s) {
    if (kp != SYS_KP_KAHAN || mode == 2) return cudaErrorInvalidValue;
    const bool save = mode == 1;
    if (wi <= 128) {
        if (dtype == BF_BF16)
            return save ? sys_launch_one<6, false, true, true, 128, __nv_bfloat16>(p, wi, gx, gy, s)
                        : sys_launch_one<6, false, false, true, 128, __nv_bfloat16>(p, wi, gx, gy, s);
        return save ? sys_launch_one<6, false, true, true, 128, float>(p, wi, gx, gy, s)
                    : sys_launch_one<6, false, false, true, 128, float>(p, wi, gx, gy, s);
    }
    if (dtype == BF_BF16)
        return save ? sys_launch_one<6, false, true, true, 256, __nv_bfloat16>(p, wi, gx, gy, s)
                    : sys_launch_one<6, false, false, true, 256, __nv_bfloat16>(p, wi, gx, gy, s);
    return save ? sys_launch_one<6, false, true, true, 256, float>(p, wi, gx, gy, s)
                : sys_launch_one<6, false, false, true, 256, float>(p, wi, gx, gy, s);
}

}  // namespace bf
