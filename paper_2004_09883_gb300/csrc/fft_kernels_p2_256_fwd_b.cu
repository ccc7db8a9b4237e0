// fft_kernels_p2_256_fwd_b.cu -- 256-thread power-of-two line passes, forward (exponent sign -1),
// layouts: kIoNC kIoCCP.
#include "fft_p2.cuh"

namespace fbfft {

LineKernel line_kernel_p2_256_fwd_b(int lg, int io)
{
    switch (lg * 4 + io) {
    case 1 * 4 + kIoNC: return p2_entry<256, true, 1, kIoNC>();
    case 1 * 4 + kIoCCP: return p2_entry<256, true, 1, kIoCCP>();
    case 2 * 4 + kIoNC: return p2_entry<256, true, 2, kIoNC>();
    case 2 * 4 + kIoCCP: return p2_entry<256, true, 2, kIoCCP>();
    case 3 * 4 + kIoNC: return p2_entry<256, true, 3, kIoNC>();
    case 3 * 4 + kIoCCP: return p2_entry<256, true, 3, kIoCCP>();
    case 4 * 4 + kIoNC: return p2_entry<256, true, 4, kIoNC>();
    case 4 * 4 + kIoCCP: return p2_entry<256, true, 4, kIoCCP>();
    case 5 * 4 + kIoNC: return p2_entry<256, true, 5, kIoNC>();
    case 5 * 4 + kIoCCP: return p2_entry<256, true, 5, kIoCCP>();
    case 6 * 4 + kIoNC: return p2_entry<256, true, 6, kIoNC>();
    case 6 * 4 + kIoCCP: return p2_entry<256, true, 6, kIoCCP>();
    case 7 * 4 + kIoNC: return p2_entry<256, true, 7, kIoNC>();
    case 7 * 4 + kIoCCP: return p2_entry<256, true, 7, kIoCCP>();
    case 8 * 4 + kIoNC: return p2_entry<256, true, 8, kIoNC>();
    case 8 * 4 + kIoCCP: return p2_entry<256, true, 8, kIoCCP>();
    case 9 * 4 + kIoNC: return p2_entry<256, true, 9, kIoNC>();
    case 9 * 4 + kIoCCP: return p2_entry<256, true, 9, kIoCCP>();
    case 10 * 4 + kIoNC: return p2_entry<256, true, 10, kIoNC>();
    case 10 * 4 + kIoCCP: return p2_entry<256, true, 10, kIoCCP>();
    case 11 * 4 + kIoNC: return p2_entry<256, true, 11, kIoNC>();
    case 11 * 4 + kIoCCP: return p2_entry<256, true, 11, kIoCCP>();
    case 12 * 4 + kIoNC: return p2_entry<256, true, 12, kIoNC>();
    case 12 * 4 + kIoCCP: return p2_entry<256, true, 12, kIoCCP>();
    default: return LineKernel{nullptr, 0, false, 0, 0};
    }
}

}  // namespace fbfft
