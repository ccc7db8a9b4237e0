// fft_kernels_plane.cu -- plane-pass kernels (fft_plane.cuh) for planes of
// 128 or 256 rows by 128 or 256 values, both directions, 512 compute threads
// (one CTA per SM) and, where the cluster stays within 8 CTAs, 256 (two).
#include "fft_plane.cuh"

namespace fbfft {

LineKernel line_kernel_plane(bool forward, int lg1, int lg2, int threads)
{
    const int key = (lg1 * 16 + lg2) * 1024 + threads;
    switch (key) {
    case (8 * 16 + 7) * 1024 + 512: return forward ? plane_entry<8, 7, 512, true>() : plane_entry<8, 7, 512, false>();
    case (7 * 16 + 7) * 1024 + 512: return forward ? plane_entry<7, 7, 512, true>() : plane_entry<7, 7, 512, false>();
    case (8 * 16 + 8) * 1024 + 512: return forward ? plane_entry<8, 8, 512, true>() : plane_entry<8, 8, 512, false>();
    case (7 * 16 + 8) * 1024 + 512: return forward ? plane_entry<7, 8, 512, true>() : plane_entry<7, 8, 512, false>();
    case (8 * 16 + 7) * 1024 + 256: return forward ? plane_entry<8, 7, 256, true>() : plane_entry<8, 7, 256, false>();
    case (7 * 16 + 7) * 1024 + 256: return forward ? plane_entry<7, 7, 256, true>() : plane_entry<7, 7, 256, false>();
    case (7 * 16 + 8) * 1024 + 256: return forward ? plane_entry<7, 8, 256, true>() : plane_entry<7, 8, 256, false>();
    default: return LineKernel{nullptr, 0, false, 0, 0};
    }
}

long long plane_smem_bytes(int lg1, int lg2, int threads)
{
    const int key = (lg1 * 16 + lg2) * 1024 + threads;
    switch (key) {
    case (8 * 16 + 7) * 1024 + 512: return PlaneCfg<8, 7, 512>::SMEM;
    case (7 * 16 + 7) * 1024 + 512: return PlaneCfg<7, 7, 512>::SMEM;
    case (8 * 16 + 8) * 1024 + 512: return PlaneCfg<8, 8, 512>::SMEM;
    case (7 * 16 + 8) * 1024 + 512: return PlaneCfg<7, 8, 512>::SMEM;
    case (8 * 16 + 7) * 1024 + 256: return PlaneCfg<8, 7, 256>::SMEM;
    case (7 * 16 + 7) * 1024 + 256: return PlaneCfg<7, 7, 256>::SMEM;
    case (7 * 16 + 8) * 1024 + 256: return PlaneCfg<7, 8, 256>::SMEM;
    default: return 0;
    }
}

}  // namespace fbfft
