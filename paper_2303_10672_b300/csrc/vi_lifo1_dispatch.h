// vi_lifo1_dispatch.h -- entry points of the LIFO lead-time-one sweep units.
#pragma once

#include "vi_kernels.h"

namespace vib {

cudaError_t describe_lifo1_d16(const KernelParams &kp, LaunchDesc &d);   // dmax < 16
cudaError_t describe_lifo1_d32(const KernelParams &kp, LaunchDesc &d);   // dmax < 32

}  // namespace vib
