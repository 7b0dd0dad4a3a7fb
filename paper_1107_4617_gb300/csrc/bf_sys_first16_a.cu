// First-chunk engine instantiations (see bf_sys_first.cuh), 128-thread strips, BF16 input
// (forward modes): pair counts 1 2 3 4 5.
#include "bf_sys_first.cuh"

namespace bf {
template cudaError_t sys_first_kp<1, 128, __nv_bfloat16>(const SysParams&, int, bool, int, int,
                                                         int, int, cudaStream_t);
template cudaError_t sys_first_kp<2, 128, __nv_bfloat16>(const SysParams&, int, bool, int, int,
                                                         int, int, cudaStream_t);
template cudaError_t sys_first_kp<3, 128, __nv_bfloat16>(const SysParams&, int, bool, int, int,
                                                         int, int, cudaStream_t);
template cudaError_t sys_first_kp<4, 128, __nv_bfloat16>(const SysParams&, int, bool, int, int,
                                                         int, int, cudaStream_t);
template cudaError_t sys_first_kp<5, 128, __nv_bfloat16>(const SysParams&, int, bool, int, int,
                                                         int, int, cudaStream_t);
}  // namespace bf
