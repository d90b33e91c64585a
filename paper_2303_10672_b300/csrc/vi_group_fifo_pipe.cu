// vi_group_fifo_pipe.cu -- instantiations of the factorised sweep (fifo, pipe).
#include "vi_group.cuh"
#include "vi_group_dispatch.h"

namespace vib {

cudaError_t describe_group_fifo_pipe(const KernelParams &kp, int xw, LaunchDesc &d) {
    return describe_group_l<0, VK_PAIR, 1>(kp, xw, d);
}

}  // namespace vib
