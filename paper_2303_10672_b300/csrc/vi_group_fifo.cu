// vi_group_fifo.cu -- instantiations of the factorised sweep (fifo).
#include "vi_group.cuh"
#include "vi_group_dispatch.h"

namespace vib {

cudaError_t describe_group_fifo(const KernelParams &kp, int xw, LaunchDesc &d) {
    return describe_group_l<0, VK_PAIR, 0>(kp, xw, d);
}

}  // namespace vib
