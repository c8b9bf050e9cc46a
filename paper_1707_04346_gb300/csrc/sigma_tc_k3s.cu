// Instantiations of the tensor-core sigma kernel for 3 bf16 slices with the A
// operand in shared memory (one translation unit per variant so that
// they compile in parallel).
#include "sigma_tc_kernel.cuh"

namespace fci {

template <int EPI>
static void *pick(int kpad) {
    switch (kpad) {
        case 16: return (void *)tc::k_sigma3_tc<3, 16, EPI, false>;
        case 32: return (void *)tc::k_sigma3_tc<3, 32, EPI, false>;
        case 48: return (void *)tc::k_sigma3_tc<3, 48, EPI, false>;
        case 64: return (void *)tc::k_sigma3_tc<3, 64, EPI, false>;
        case 80: return (void *)tc::k_sigma3_tc<3, 80, EPI, false>;
        case 96: return (void *)tc::k_sigma3_tc<3, 96, EPI, false>;
        default: return nullptr;
    }
}

void *tc_kernel_3s(int kpad, int epi) {
    return epi == 4 ? pick<4>(kpad) : epi == 3 ? pick<3>(kpad) : pick<2>(kpad);
}

}  // namespace fci
