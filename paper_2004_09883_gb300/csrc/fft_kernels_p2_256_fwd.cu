// fft_kernels_p2_256_fwd.cu -- 256-thread line passes with compile-time
// power-of-two schedules, forward (exponent sign -1).
#include "fft_device.cuh"

namespace fbfft {

LineKernel line_kernel_p2_256_fwd(int lg)
{
    switch (lg) {
    case 1: return kernel_entry<256, true, 1>();
    case 2: return kernel_entry<256, true, 2>();
    case 3: return kernel_entry<256, true, 3>();
    case 4: return kernel_entry<256, true, 4>();
    case 5: return kernel_entry<256, true, 5>();
    case 6: return kernel_entry<256, true, 6>();
    case 7: return kernel_entry<256, true, 7>();
    case 8: return kernel_entry<256, true, 8>();
    case 9: return kernel_entry<256, true, 9>();
    case 10: return kernel_entry<256, true, 10>();
    case 11: return kernel_entry<256, true, 11>();
    case 12: return kernel_entry<256, true, 12>();
    default: return LineKernel{nullptr, nullptr, nullptr};
    }
}

}  // namespace fbfft
