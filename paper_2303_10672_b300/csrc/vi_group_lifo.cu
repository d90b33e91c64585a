// vi_group_lifo.cu -- instantiations of the factorised sweep (lifo).
#include "vi_group.cuh"
#include "vi_group_dispatch.h"

namespace vib {

cudaError_t describe_group_lifo(const KernelParams &kp, int xw, LaunchDesc &d) {
    return describe_group_l<1, VK_PAIR, 0>(kp, xw, d);
}

}  // namespace vib
