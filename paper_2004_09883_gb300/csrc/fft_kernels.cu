// fft_kernels.cu -- the generic line-pass kernel and the kernel dispatch table.
#include "fft_device.cuh"

namespace fbfft {

LineKernel line_kernel_generic(bool forward)
{
    return forward ? kernel_entry<kGenericThreads, true, 0>() : kernel_entry<kGenericThreads, false, 0>();
}

LineKernel line_kernel(int threads, bool forward, int lg)
{
    if (lg == 0) return threads == kGenericThreads ? line_kernel_generic(forward) : LineKernel{nullptr, nullptr, nullptr};
    if (lg < 0 || lg > kMaxLineLog2) return LineKernel{nullptr, nullptr, nullptr};
    if (threads == 256) return forward ? line_kernel_p2_256_fwd(lg) : line_kernel_p2_256_inv(lg);
    if (threads == 512) return line_kernel_p2_512(forward, lg);
    return LineKernel{nullptr, nullptr, nullptr};
}

}  // namespace fbfft
