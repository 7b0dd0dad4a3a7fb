// First-chunk engine instantiations (see bf_sys_first.cuh), 64-thread strips: pair counts 11.
#include "bf_sys_first.cuh"

namespace bf {
template cudaError_t sys_first_kp<11, 64, float>(const SysParams&, int, bool, int, int, int,
                                                 int, cudaStream_t);
}  // namespace bf
