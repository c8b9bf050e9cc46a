// Instantiations of the tensor-core sigma kernel for 3 bf16 slices with the A
// operand in tensor memory (one translation unit per variant so that
// they compile in parallel).
#include "sigma_tc_kernel.cuh"

namespace fci {

template <int EPI>
static void *pick(int kpad) {
    switch (kpad) {
        case 16: return (void *)tc::k_sigma3_tc<3, 16, EPI, true>;
        case 32: return (void *)tc::k_sigma3_tc<3, 32, EPI, true>;
        case 48: return (void *)tc::k_sigma3_tc<3, 48, EPI, true>;
        case 64: return (void *)tc::k_sigma3_tc<3, 64, EPI, true>;
        case 80: return (void *)tc::k_sigma3_tc<3, 80, EPI, true>;
        case 96: return (void *)tc::k_sigma3_tc<3, 96, EPI, true>;
        default: return nullptr;
    }
}

void *tc_kernel_3t(int kpad, int epi) {
    return epi == 4 ? pick<4>(kpad) : epi == 3 ? pick<3>(kpad) : pick<2>(kpad);
}

}  // namespace fci
