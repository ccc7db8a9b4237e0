// fft_kernels_mixed.cu -- mixed-radix line passes: the power-of-two factor's
// radices at compile time (template on its log2), then the 5s and 3s.
#include "fft_device.cuh"

namespace fbfft {

LineKernel line_kernel_mixed(bool forward, int lg2)
{
    switch (lg2) {
    case 0: return forward ? mixed_entry<true, 0>() : mixed_entry<false, 0>();
    case 1: return forward ? mixed_entry<true, 1>() : mixed_entry<false, 1>();
    case 2: return forward ? mixed_entry<true, 2>() : mixed_entry<false, 2>();
    case 3: return forward ? mixed_entry<true, 3>() : mixed_entry<false, 3>();
    case 4: return forward ? mixed_entry<true, 4>() : mixed_entry<false, 4>();
    case 5: return forward ? mixed_entry<true, 5>() : mixed_entry<false, 5>();
    case 6: return forward ? mixed_entry<true, 6>() : mixed_entry<false, 6>();
    case 7: return forward ? mixed_entry<true, 7>() : mixed_entry<false, 7>();
    case 8: return forward ? mixed_entry<true, 8>() : mixed_entry<false, 8>();
    case 9: return forward ? mixed_entry<true, 9>() : mixed_entry<false, 9>();
    default: return LineKernel{nullptr, 0, false, 0, 0, 0};
    }
}

}  // namespace fbfft
