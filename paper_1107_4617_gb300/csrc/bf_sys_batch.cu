// Persistent batch launches of the three groups (bf_sys_batch.cuh).
#include "bf_sys_batch.cuh"

namespace bf {

int sys_batch_kind(int K, int kstart, int* group) {
    // odd N: K harmonics in pairs; even N: the constant harmonic apart
    if (kstart == 0 && K < 2) return -1;
    const int np = kstart == 1 ? K : K - 1;
    const int kp = (np + 1) / 2;
    const int seed = kstart == 1 ? 1 : 2;
    if (kp <= SYS_BATCH_SMALL_KP) {
        *group = 0;
        return ((seed - 1) * SYS_BATCH_SMALL_KP + kp - 1) * 2 + (np & 1);
    }
    return -1;
}

int sys_batch_grid(int group, int in_dtype) {
    const bool h = in_dtype == BF_BF16;
    if (group == 0) return h ? batch_grid<128, __nv_bfloat16, 1>() : batch_grid<128, float, 1>();
    if (group == 1) return h ? batch_grid<128, __nv_bfloat16, 0>() : batch_grid<128, float, 0>();
    return h ? batch_grid<256, __nv_bfloat16, 0>() : batch_grid<256, float, 0>();
}

cudaError_t launch_sys_batch(SysBatchTable* tab, int group, int grid, int in_dtype,
                             cudaStream_t s) {
    const bool h = in_dtype == BF_BF16;
    if (group == 0)
        return h ? batch_launch<128, __nv_bfloat16, 1>(tab, group, grid, s)
                 : batch_launch<128, float, 1>(tab, group, grid, s);
    if (group == 1)
        return h ? batch_launch<128, __nv_bfloat16, 0>(tab, group, grid, s)
                 : batch_launch<128, float, 0>(tab, group, grid, s);
    return h ? batch_launch<256, __nv_bfloat16, 0>(tab, group, grid, s)
             : batch_launch<256, float, 0>(tab, group, grid, s);
}

}  // namespace bf
