// fft_kernels_p2_256_inv_a.cu -- 256-thread power-of-two line passes, inverse (exponent sign +1),
// layouts: kIoNN kIoCC.
#include "fft_p2.cuh"

namespace fbfft {

LineKernel line_kernel_p2_256_inv_a(int lg, int io)
{
    switch (lg * 4 + io) {
    case 1 * 4 + kIoNN: return p2_entry<256, false, 1, kIoNN>();
    case 1 * 4 + kIoCC: return p2_entry<256, false, 1, kIoCC>();
    case 2 * 4 + kIoNN: return p2_entry<256, false, 2, kIoNN>();
    case 2 * 4 + kIoCC: return p2_entry<256, false, 2, kIoCC>();
    case 3 * 4 + kIoNN: return p2_entry<256, false, 3, kIoNN>();
    case 3 * 4 + kIoCC: return p2_entry<256, false, 3, kIoCC>();
    case 4 * 4 + kIoNN: return p2_entry<256, false, 4, kIoNN>();
    case 4 * 4 + kIoCC: return p2_entry<256, false, 4, kIoCC>();
    case 5 * 4 + kIoNN: return p2_entry<256, false, 5, kIoNN>();
    case 5 * 4 + kIoCC: return p2_entry<256, false, 5, kIoCC>();
    case 6 * 4 + kIoNN: return p2_entry<256, false, 6, kIoNN>();
    case 6 * 4 + kIoCC: return p2_entry<256, false, 6, kIoCC>();
    case 7 * 4 + kIoNN: return p2_entry<256, false, 7, kIoNN>();
    case 7 * 4 + kIoCC: return p2_entry<256, false, 7, kIoCC>();
    case 8 * 4 + kIoNN: return p2_entry<256, false, 8, kIoNN>();
    case 8 * 4 + kIoCC: return p2_entry<256, false, 8, kIoCC>();
    case 9 * 4 + kIoNN: return p2_entry<256, false, 9, kIoNN>();
    case 9 * 4 + kIoCC: return p2_entry<256, false, 9, kIoCC>();
    case 10 * 4 + kIoNN: return p2_entry<256, false, 10, kIoNN>();
    case 10 * 4 + kIoCC: return p2_entry<256, false, 10, kIoCC>();
    case 11 * 4 + kIoNN: return p2_entry<256, false, 11, kIoNN>();
    case 11 * 4 + kIoCC: return p2_entry<256, false, 11, kIoCC>();
    case 12 * 4 + kIoNN: return p2_entry<256, false, 12, kIoNN>();
    case 12 * 4 + kIoCC: return p2_entry<256, false, 12, kIoCC>();
    default: return LineKernel{nullptr, 0, false, 0, 0};
    }
}

}  // namespace fbfft
