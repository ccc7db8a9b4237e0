// fft_kernels_uneven.cu -- k_fft_uneven (one kernel per direction) with its
// launch and occupancy helpers.
#include <cstdlib>

#include "fft_uneven.cuh"

namespace fbfft {

namespace {
using UnevenFn = void (*)(UnevenArgs);
UnevenFn uneven_fn(bool forward) { return forward ? k_fft_uneven<true> : k_fft_uneven<false>; }
UnevenFn uneven_one_fn(bool forward) { return forward ? k_fft_uneven_one<true> : k_fft_uneven_one<false>; }
using UnevenInlineFn = void (*)(UnevenInlineArgs);
UnevenInlineFn uneven_inline_fn(bool forward)
{
    return forward ? k_fft_uneven_inline<true> : k_fft_uneven_inline<false>;
}
}  // namespace

cudaError_t uneven_launch_inline(bool forward, const UnevenInlineArgs& a, long long grid, size_t smem,
                                 cudaStream_t stream)
{
    if (grid <= 0) return cudaSuccess;
    const UnevenInlineFn fn = uneven_inline_fn(forward);
    cudaError_t e = kernel_smem_optin((const void*)fn, 0);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3(kUnevenThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = stream;
    cfg.numAttrs = 0;
    return cudaLaunchKernelEx(&cfg, fn, a);
}

cudaError_t uneven_occupancy_inline(bool forward, size_t smem, int* blocks_per_sm)
{
    const UnevenInlineFn fn = uneven_inline_fn(forward);
    cudaError_t e = kernel_smem_optin((const void*)fn, 0);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, (const void*)fn, kUnevenThreads, smem);
}

cudaError_t uneven_launch(bool forward, const UnevenArgs& a, long long grid, size_t smem, cudaStream_t stream)
{
    if (grid <= 0) return cudaSuccess;
    const UnevenFn fn = uneven_fn(forward);
    cudaError_t e = kernel_smem_optin((const void*)fn, 0);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3(kUnevenThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = stream;
    cfg.numAttrs = 0;
    return cudaLaunchKernelEx(&cfg, fn, a);
}

cudaError_t uneven_occupancy(bool forward, size_t smem, int* blocks_per_sm)
{
    const UnevenFn fn = uneven_fn(forward);
    cudaError_t e = kernel_smem_optin((const void*)fn, 0);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, (const void*)fn, kUnevenThreads, smem);
}

cudaError_t uneven_launch_one(bool forward, const UnevenArgs& a, long long grid, size_t smem, cudaStream_t stream)
{
    if (grid <= 0) return cudaSuccess;
    const UnevenFn fn = uneven_one_fn(forward);
    cudaError_t e = kernel_smem_optin((const void*)fn, 0);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3(kUnevenThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = stream;
    cfg.numAttrs = 0;
    return cudaLaunchKernelEx(&cfg, fn, a);
}

cudaError_t uneven_occupancy_one(bool forward, size_t smem, int* blocks_per_sm)
{
    const UnevenFn fn = uneven_one_fn(forward);
    cudaError_t e = kernel_smem_optin((const void*)fn, 0);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, (const void*)fn, kUnevenThreads, smem);
}

}  // namespace fbfft
