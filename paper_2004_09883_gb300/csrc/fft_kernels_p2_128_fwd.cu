// fft_kernels_p2_128_fwd.cu -- 128-thread power-of-two line passes, forward (exponent sign -1):
// contiguous lines of length 32 ... 256 with three landing buffers per CTA
// (and the 64-thread variant).
#include "fft_p2.cuh"

namespace fbfft {

LineKernel line_kernel_p2_128_fwd(int lg, int io)
{
    if (io != kIoNN) return LineKernel{nullptr, 0, false, 0, 0};
    switch (lg) {
    case 5: return p2_entry<128, true, 5, kIoNN>();
    case 6: return p2_entry<128, true, 6, kIoNN>();
    case 7: return p2_entry<128, true, 7, kIoNN>();
    case 8: return p2_entry<128, true, 8, kIoNN>();
    default: return LineKernel{nullptr, 0, false, 0, 0};
    }
}

LineKernel line_kernel_p2_64_fwd(int lg, int io)
{
    if (io != kIoNN) return LineKernel{nullptr, 0, false, 0, 0};
    switch (lg) {
    case 5: return p2_entry<64, true, 5, kIoNN>();
    case 6: return p2_entry<64, true, 6, kIoNN>();
    case 7: return p2_entry<64, true, 7, kIoNN>();
    case 8: return p2_entry<64, true, 8, kIoNN>();
    default: return LineKernel{nullptr, 0, false, 0, 0};
    }
}

}  // namespace fbfft
