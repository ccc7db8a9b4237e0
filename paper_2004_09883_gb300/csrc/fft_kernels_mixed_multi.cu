// fft_kernels_mixed_multi.cu -- the mixed line pass over several jobs in one
// launch (k_fft_mixed_multi), one kernel per direction and power-of-two factor,
// with its launch and occupancy helpers.
#include <cstdlib>

#include "fft_device.cuh"

namespace fbfft {

namespace {

using MultiFn = void (*)(MultiArgs);

template <bool FWD>
MultiFn multi_fn(int lg2)
{
    switch (lg2) {
    case 0: return k_fft_mixed_multi<kMixedThreads, FWD, 0>;
    case 1: return k_fft_mixed_multi<kMixedThreads, FWD, 1>;
    case 2: return k_fft_mixed_multi<kMixedThreads, FWD, 2>;
    case 3: return k_fft_mixed_multi<kMixedThreads, FWD, 3>;
    case 4: return k_fft_mixed_multi<kMixedThreads, FWD, 4>;
    case 5: return k_fft_mixed_multi<kMixedThreads, FWD, 5>;
    case 6: return k_fft_mixed_multi<kMixedThreads, FWD, 6>;
    case 7: return k_fft_mixed_multi<kMixedThreads, FWD, 7>;
    case 8: return k_fft_mixed_multi<kMixedThreads, FWD, 8>;
    case 9: return k_fft_mixed_multi<kMixedThreads, FWD, 9>;
    default: return nullptr;
    }
}

// Opt-in dynamic shared memory, once per (kernel, device).
cudaError_t prepare(MultiFn fn) { return kernel_smem_optin((const void*)fn, 0); }

bool pdl_on()
{
    static const bool v = [] {
        const char* s = std::getenv("FB_FFT_PDL");
        return !(s && s[0] == '0');
    }();
    return v;
}

}  // namespace

cudaError_t mixed_multi_occupancy(bool forward, int lg2, size_t smem, int* blocks_per_sm)
{
    const MultiFn fn = forward ? multi_fn<true>(lg2) : multi_fn<false>(lg2);
    if (!fn) return cudaErrorInvalidValue;
    cudaError_t e = prepare(fn);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, (const void*)fn, kMixedThreads, smem);
}

cudaError_t mixed_multi_launch(bool forward, int lg2, const MultiArgs& a, long long grid, size_t smem,
                               cudaStream_t stream)
{
    const MultiFn fn = forward ? multi_fn<true>(lg2) : multi_fn<false>(lg2);
    if (!fn) return cudaErrorInvalidValue;
    if (grid <= 0 || a.njobs <= 0) return cudaSuccess;
    cudaError_t e = prepare(fn);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(grid > 0x7fffffffLL ? 0x7fffffffLL : grid));
    cfg.blockDim = dim3(kMixedThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = pdl_on() ? 1 : 0;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, fn, a);
}

}  // namespace fbfft
