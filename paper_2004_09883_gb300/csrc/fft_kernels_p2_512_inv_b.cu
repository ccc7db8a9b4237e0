// fft_kernels_p2_512_inv_b.cu -- 512-thread power-of-two line passes, inverse (exponent sign +1),
// layouts: kIoNC kIoCCP.
#include "fft_p2.cuh"

namespace fbfft {

LineKernel line_kernel_p2_512_inv_b(int lg, int io)
{
    switch (lg * 4 + io) {
    case 9 * 4 + kIoNC: return p2_entry<512, false, 9, kIoNC>();
    case 9 * 4 + kIoCCP: return p2_entry<512, false, 9, kIoCCP>();
    case 10 * 4 + kIoNC: return p2_entry<512, false, 10, kIoNC>();
    case 10 * 4 + kIoCCP: return p2_entry<512, false, 10, kIoCCP>();
    case 11 * 4 + kIoNC: return p2_entry<512, false, 11, kIoNC>();
    case 11 * 4 + kIoCCP: return p2_entry<512, false, 11, kIoCCP>();
    case 12 * 4 + kIoNC: return p2_entry<512, false, 12, kIoNC>();
    case 12 * 4 + kIoCCP: return p2_entry<512, false, 12, kIoCCP>();
    default: return LineKernel{nullptr, 0, false, 0, 0};
    }
}

}  // namespace fbfft
