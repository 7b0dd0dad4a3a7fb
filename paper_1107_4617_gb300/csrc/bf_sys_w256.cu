// Instantiations of the skewed-strip engine for strips of up to 256 threads.
#include "bf_sys_engine.cuh"

namespace bf {

#define BF_SYS_MODES(KP, T)                                                               \
    if (mode == 2) return sys_launch_one<KP, true, false, false, 256, T, false, 0, 1>(p, wi, gx, gy, s); \
    if (mode == 1) return sys_launch_one<KP, false, true, false, 256, T>(p, wi, gx, gy, s); \
    return sys_launch_one<KP, false, false, false, 256, T>(p, wi, gx, gy, s);
#define BF_SYS_CASE(KP)                              \
    case KP:                                         \
        if (dtype == BF_BF16) {                      \
            BF_SYS_MODES(KP, __nv_bfloat16)          \
        } else {                                     \
            BF_SYS_MODES(KP, float)                  \
        }

cudaError_t launch_sys_w256(const SysParams& p, int mode, int dtype, int kp, int wi, int gx,
                            int gy, cudaStream_t s) {
    switch (kp) {
        BF_SYS_CASE(1)
        BF_SYS_CASE(2)
        BF_SYS_CASE(3)
        BF_SYS_CASE(4)
        BF_SYS_CASE(6)
        BF_SYS_CASE(8)
        BF_SYS_CASE(11)
    }
    return cudaErrorInvalidValue;
}

}  // namespace bf
