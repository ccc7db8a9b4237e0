// fft_kernels_p2tc_inv.cu -- power-of-two line passes with radix-16 stages on the tensor
// cores, inverse (exponent sign +1): L = 256 ... 4096, every layout, 256 compute
// threads (two CTAs per SM, so one computes while the other waits on its products).
#include "fft_p2.cuh"

namespace fbfft {

LineKernel line_kernel_p2tc_inv(int threads, int lg, int io)
{
    if (threads != 256) return LineKernel{nullptr, 0, false, 0, 0};
    switch (lg * 4 + io) {
    case 8 * 4 + kIoNN: return p2_entry<256, false, 8, kIoNN, true>();
    case 8 * 4 + kIoCC: return p2_entry<256, false, 8, kIoCC, true>();
    case 8 * 4 + kIoNC: return p2_entry<256, false, 8, kIoNC, true>();
    case 8 * 4 + kIoCCP: return p2_entry<256, false, 8, kIoCCP, true>();
    case 9 * 4 + kIoNN: return p2_entry<256, false, 9, kIoNN, true>();
    case 9 * 4 + kIoCC: return p2_entry<256, false, 9, kIoCC, true>();
    case 9 * 4 + kIoNC: return p2_entry<256, false, 9, kIoNC, true>();
    case 9 * 4 + kIoCCP: return p2_entry<256, false, 9, kIoCCP, true>();
    case 10 * 4 + kIoNN: return p2_entry<256, false, 10, kIoNN, true>();
    case 10 * 4 + kIoCC: return p2_entry<256, false, 10, kIoCC, true>();
    case 10 * 4 + kIoNC: return p2_entry<256, false, 10, kIoNC, true>();
    case 10 * 4 + kIoCCP: return p2_entry<256, false, 10, kIoCCP, true>();
    case 11 * 4 + kIoNN: return p2_entry<256, false, 11, kIoNN, true>();
    case 11 * 4 + kIoCC: return p2_entry<256, false, 11, kIoCC, true>();
    case 11 * 4 + kIoNC: return p2_entry<256, false, 11, kIoNC, true>();
    case 11 * 4 + kIoCCP: return p2_entry<256, false, 11, kIoCCP, true>();
    case 12 * 4 + kIoNN: return p2_entry<256, false, 12, kIoNN, true>();
    case 12 * 4 + kIoCC: return p2_entry<256, false, 12, kIoCC, true>();
    case 12 * 4 + kIoNC: return p2_entry<256, false, 12, kIoNC, true>();
    case 12 * 4 + kIoCCP: return p2_entry<256, false, 12, kIoCCP, true>();
    default: return LineKernel{nullptr, 0, false, 0, 0};
    }
}

}  // namespace fbfft
