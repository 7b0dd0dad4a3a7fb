// First-chunk engine instantiations (see bf_sys_first.cuh), 128-thread strips, BF16 input
// (forward modes): pair counts 10.
#include "bf_sys_first.cuh"

namespace bf {
template cudaError_t sys_first_kp<10, 128, __nv_bfloat16>(const SysParams&, int, bool, int, int,
                                                         int, int, cudaStream_t);
}  // namespace bf
