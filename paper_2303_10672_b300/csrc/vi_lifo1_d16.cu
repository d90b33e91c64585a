// vi_lifo1_d16.cu -- instantiations of the LIFO lead-time-one sweep with a pmf of
// at most 16 entries (dmax < 16), one per radix G = Q+1 in 2..16.
#include "vi_lifo1.cuh"
#include "vi_lifo1_dispatch.h"

namespace vib {

cudaError_t describe_lifo1_d16(const KernelParams &kp, LaunchDesc &d) {
    switch (kp.p[0].G) {
#define VIB_G(g) \
    case g: return describe_lifo1_t<g, 16>(kp, d);
        VIB_G(2) VIB_G(3) VIB_G(4) VIB_G(5) VIB_G(6) VIB_G(7) VIB_G(8) VIB_G(9) VIB_G(10) VIB_G(11)
        VIB_G(12) VIB_G(13) VIB_G(14) VIB_G(15) VIB_G(16)
#undef VIB_G
        default: return cudaErrorInvalidValue;
    }
}

// one product, float-pair values, LIFO, lead time one, at least one stock slot
// besides the expiring one's (m >= 2), 2 <= Q+1 <= 16 and dmax < 32
bool lifo1_supported(const KernelParams &kp, int vk, int kahan) {
    const ProdParams &P = kp.p[0];
    return kp.n_products == 1 && vk == VK_PAIR && !kahan && kp.issuing == 1 && P.L == 1 && P.m >= 2 &&
           P.G >= 2 && P.G <= 16 && P.dmax < 32 && !kp.pc && P.off_LF > 0;
}

cudaError_t describe_lifo1(const KernelParams &kp, LaunchDesc &d) {
    d.n_pre = 0;
    return kp.p[0].dmax < 16 ? describe_lifo1_d16(kp, d) : describe_lifo1_d32(kp, d);
}

}  // namespace vib
