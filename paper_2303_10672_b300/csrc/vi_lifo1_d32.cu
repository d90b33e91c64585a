// vi_lifo1_d32.cu -- instantiations of the LIFO lead-time-one sweep with a pmf of
// at most 32 entries (dmax < 32), one per radix G = Q+1 in 2..16.
#include "vi_lifo1.cuh"
#include "vi_lifo1_dispatch.h"

namespace vib {

cudaError_t describe_lifo1_d32(const KernelParams &kp, LaunchDesc &d) {
    switch (kp.p[0].G) {
#define VIB_G(g) \
    case g: return describe_lifo1_t<g, 32>(kp, d);
        VIB_G(2) VIB_G(3) VIB_G(4) VIB_G(5) VIB_G(6) VIB_G(7) VIB_G(8) VIB_G(9) VIB_G(10) VIB_G(11)
        VIB_G(12) VIB_G(13) VIB_G(14) VIB_G(15) VIB_G(16)
#undef VIB_G
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace vib
