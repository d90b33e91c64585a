// vi_group_dispatch.h -- entry points of the per-variant translation units.
#pragma once

#include "vi_kernels.h"

namespace vib {

cudaError_t describe_group_fifo(const KernelParams &kp, int xw, LaunchDesc &d);        // pairs, L = 1
cudaError_t describe_group_fifo_pipe(const KernelParams &kp, int xw, LaunchDesc &d);   // pairs, L >= 2
cudaError_t describe_group_lifo(const KernelParams &kp, int xw, LaunchDesc &d);
cudaError_t describe_group_lifo_pipe(const KernelParams &kp, int xw, LaunchDesc &d);
cudaError_t describe_group_fifo_single(const KernelParams &kp, int xw, LaunchDesc &d); // single floats
cudaError_t describe_group_lifo_single(const KernelParams &kp, int xw, LaunchDesc &d);

}  // namespace vib
