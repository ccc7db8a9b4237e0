// fft_kernels_p2_512.cu -- 512-thread line passes with compile-time
// power-of-two schedules for 512 <= L <= 4096 (wider tiles for strided axes).
#include "fft_device.cuh"

namespace fbfft {

LineKernel line_kernel_p2_512(bool forward, int lg)
{
    switch (lg) {
    case 9: return forward ? kernel_entry<512, true, 9>() : kernel_entry<512, false, 9>();
    case 10: return forward ? kernel_entry<512, true, 10>() : kernel_entry<512, false, 10>();
    case 11: return forward ? kernel_entry<512, true, 11>() : kernel_entry<512, false, 11>();
    case 12: return forward ? kernel_entry<512, true, 12>() : kernel_entry<512, false, 12>();
    default: return LineKernel{nullptr, nullptr, nullptr};
    }
}

}  // namespace fbfft
