// fft_kernels_p2_256_inv.cu -- 256-thread line passes with compile-time
// power-of-two schedules, inverse (exponent sign +1).
#include "fft_device.cuh"

namespace fbfft {

LineKernel line_kernel_p2_256_inv(int lg)
{
    switch (lg) {
    case 1: return kernel_entry<256, false, 1>();
    case 2: return kernel_entry<256, false, 2>();
    case 3: return kernel_entry<256, false, 3>();
    case 4: return kernel_entry<256, false, 4>();
    case 5: return kernel_entry<256, false, 5>();
    case 6: return kernel_entry<256, false, 6>();
    case 7: return kernel_entry<256, false, 7>();
    case 8: return kernel_entry<256, false, 8>();
    case 9: return kernel_entry<256, false, 9>();
    case 10: return kernel_entry<256, false, 10>();
    case 11: return kernel_entry<256, false, 11>();
    case 12: return kernel_entry<256, false, 12>();
    default: return LineKernel{nullptr, nullptr, nullptr};
    }
}

}  // namespace fbfft
