// vi_group_lifo_pipe.cu -- instantiations of the factorised sweep (lifo, pipe).
#include "vi_group.cuh"
#include "vi_group_dispatch.h"

namespace vib {

cudaError_t describe_group_lifo_pipe(const KernelParams &kp, int xw, LaunchDesc &d) {
    return describe_group_l<1, VK_PAIR, 1>(kp, xw, d);
}

}  // namespace vib
