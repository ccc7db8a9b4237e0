// fft_kernels_p2_512_fwd_a.cu -- 512-thread power-of-two line passes, forward (exponent sign -1),
// layouts: kIoCC.
#include "fft_p2.cuh"

namespace fbfft {

LineKernel line_kernel_p2_512_fwd_a(int lg, int io)
{
    switch (lg * 4 + io) {
    case 9 * 4 + kIoCC: return p2_entry<512, true, 9, kIoCC>();
    case 10 * 4 + kIoCC: return p2_entry<512, true, 10, kIoCC>();
    case 11 * 4 + kIoCC: return p2_entry<512, true, 11, kIoCC>();
    case 12 * 4 + kIoCC: return p2_entry<512, true, 12, kIoCC>();
    default: return LineKernel{nullptr, 0, false, 0, 0};
    }
}

}  // namespace fbfft
