// First-chunk engine instantiations (see bf_sys_first.cuh), 64-thread strips: pair counts 8 9.
#include "bf_sys_first.cuh"

namespace bf {
template cudaError_t sys_first_kp<8, 64, float>(const SysParams&, int, bool, int, int, int,
                                                 int, cudaStream_t);
template cudaError_t sys_first_kp<9, 64, float>(const SysParams&, int, bool, int, int, int,
                                                 int, cudaStream_t);
}  // namespace bf
