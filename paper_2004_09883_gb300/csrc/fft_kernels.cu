// fft_kernels.cu -- the generic line-pass kernel, the kernel table and the
// launch path shared by all line-pass kernels.
#include <cstdint>
#include <cstdlib>
#include <mutex>

#include "fft_p2.cuh"

namespace fbfft {

LineKernel line_kernel_p2_256_fwd_a(int lg, int io);
LineKernel line_kernel_p2_256_fwd_b(int lg, int io);
LineKernel line_kernel_p2_256_inv_a(int lg, int io);
LineKernel line_kernel_p2_256_inv_b(int lg, int io);
LineKernel line_kernel_p2_512_fwd_a(int lg, int io);
LineKernel line_kernel_p2_512_fwd_b(int lg, int io);
LineKernel line_kernel_p2_512_inv_a(int lg, int io);
LineKernel line_kernel_p2_512_inv_b(int lg, int io);
LineKernel line_kernel_p2_128_fwd(int lg, int io);
LineKernel line_kernel_p2_128_inv(int lg, int io);
LineKernel line_kernel_p2_64_fwd(int lg, int io);
LineKernel line_kernel_p2_64_inv(int lg, int io);
LineKernel line_kernel_p2tc_fwd(int threads, int lg, int io);
LineKernel line_kernel_p2tc_inv(int threads, int lg, int io);

LineKernel line_kernel_generic(bool forward)
{
    return forward ? generic_entry<kGenericThreads, true>() : generic_entry<kGenericThreads, false>();
}

LineKernel line_kernel_p2(int threads, bool forward, int lg, int io)
{
    const LineKernel none{nullptr, 0, false, 0, 0};
    if (lg < 1 || lg > kMaxLineLog2 || io < kIoNN || io > kIoCCP) return none;
    const bool a = io == kIoNN || io == kIoCC;
    if (threads == 128) return forward ? line_kernel_p2_128_fwd(lg, io) : line_kernel_p2_128_inv(lg, io);
    if (threads == 64) return forward ? line_kernel_p2_64_fwd(lg, io) : line_kernel_p2_64_inv(lg, io);
    if (threads == 256)
        return forward ? (a ? line_kernel_p2_256_fwd_a(lg, io) : line_kernel_p2_256_fwd_b(lg, io))
                       : (a ? line_kernel_p2_256_inv_a(lg, io) : line_kernel_p2_256_inv_b(lg, io));
    if (threads == 512)
        return forward ? (a ? line_kernel_p2_512_fwd_a(lg, io) : line_kernel_p2_512_fwd_b(lg, io))
                       : (a ? line_kernel_p2_512_inv_a(lg, io) : line_kernel_p2_512_inv_b(lg, io));
    return none;
}

LineKernel line_kernel_p2tc(int threads, bool forward, int lg, int io)
{
    const LineKernel none{nullptr, 0, false, 0, 0};
    if (lg < 8 || lg > kMaxLineLog2 || io < kIoNN || io > kIoCCP) return none;
    return forward ? line_kernel_p2tc_fwd(threads, lg, io) : line_kernel_p2tc_inv(threads, lg, io);
}

// Kernels whose shared-memory limit is set, per device: a fixed open-addressing
// table (no heap), keyed by the kernel's address.  A full table only means
// the attribute is set again at every launch.
cudaError_t kernel_smem_optin(const void* fn, int split_regs)
{
    constexpr int kSlots = 2048;
    static std::mutex mu;
    static const void* keys[kSlots];
    static unsigned long long masks[kSlots];
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const unsigned long long bit = 1ULL << (dev & 63);
    std::lock_guard<std::mutex> g(mu);
    int slot = -1;
    for (int probe = 0, h = (int)(((uintptr_t)fn >> 4) % kSlots); probe < kSlots; ++probe, h = (h + 1) % kSlots) {
        if (keys[h] == fn || keys[h] == nullptr) {
            slot = h;
            break;
        }
    }
    if (slot >= 0 && keys[slot] == fn && (masks[slot] & bit)) return cudaSuccess;
    int optin = 0;
    e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e != cudaSuccess) return e;
    cudaFuncAttributes fa;
    e = cudaFuncGetAttributes(&fa, fn);
    if (e != cudaSuccess) return e;
    // a kernel that rebalances registers with setmaxnreg must get exactly the
    // pool its split was sized for; with fewer, setmaxnreg.inc would never return
    if (split_regs > 0 && fa.numRegs != split_regs) return cudaErrorInvalidKernelImage;
    e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - (int)fa.sharedSizeBytes);
    if (e != cudaSuccess) return e;
    if (slot >= 0) {
        keys[slot] = fn;
        masks[slot] |= bit;
    }
    return cudaSuccess;
}

namespace {
bool pdl_enabled()
{
    static const bool v = [] {
        const char* s = std::getenv("FB_FFT_PDL");
        return !(s && s[0] == '0');
    }();
    return v;
}

// The opt-in dynamic shared-memory limit is a per-device function attribute:
// set it once per (kernel, device).
cudaError_t ensure_smem_attr(const LineKernel& k) { return kernel_smem_optin((const void*)k.fn, k.split_regs); }
}  // namespace

cudaError_t line_launch(const LineKernel& k, const LineArgs& a, long long grid, size_t smem, cudaStream_t stream)
{
    if (grid <= 0) return cudaSuccess;
    cudaError_t e = ensure_smem_attr(k);
    if (e != cudaSuccess) return e;
    const unsigned g = (unsigned)(grid > 0x7fffffffLL ? 0x7fffffffLL : grid);
    // programmatic dependent launch: the kernel may start while the previous
    // pass on the stream drains (every line kernel waits for it before its
    // first global access, see pdl_start)
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(g);
    cfg.blockDim = dim3(k.threads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = stream;
    cudaLaunchAttribute attr[2];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = pdl_enabled() ? 1 : 0;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (k.cluster > 1) {  // the grid is a whole number of clusters (the planner sizes it so)
        if (g % (unsigned)k.cluster != 0) return cudaErrorInvalidConfiguration;
        attr[1].id = cudaLaunchAttributeClusterDimension;
        attr[1].val.clusterDim.x = (unsigned)k.cluster;
        attr[1].val.clusterDim.y = 1;
        attr[1].val.clusterDim.z = 1;
        cfg.numAttrs = 2;
    }
    return cudaLaunchKernelEx(&cfg, k.fn, a);
}

cudaError_t line_cluster_occupancy(const LineKernel& k, size_t smem, int* clusters)
{
    *clusters = 0;
    cudaError_t e = ensure_smem_attr(k);
    if (e != cudaSuccess) return e;
    const int cs = k.cluster > 1 ? k.cluster : 1;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)cs);
    cfg.blockDim = dim3(k.threads);
    cfg.dynamicSmemBytes = smem;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)cs;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaOccupancyMaxActiveClusters(clusters, (const void*)k.fn, &cfg);
}

cudaError_t line_occupancy(const LineKernel& k, size_t smem, int* blocks_per_sm)
{
    cudaError_t e = ensure_smem_attr(k);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, (const void*)k.fn, k.threads, smem);
}

void line_kernel_name(const LineKernel& k, char* buf, size_t n)
{
    static const char* io_names[4] = {"NN", "CC", "NC", "CCP"};
    if (k.kind == 3)
        snprintf(buf, n, "k_fft_plane<%dx%d,%s>", 1 << k.lg1, 1 << k.lg, k.fwd ? "fwd" : "inv");
    else if (k.kind == 2)
        snprintf(buf, n, "k_fft_mixed<%d,%s,2^%d>", k.threads, k.fwd ? "fwd" : "inv", k.lg);
    else if (k.kind == 0)
        snprintf(buf, n, "k_fft_p2%s<%d,%s,L=%d,%s>", k.tc ? "tc" : "", k.threads - k.producers, k.fwd ? "fwd" : "inv", 1 << k.lg,
                 (k.io >= 0 && k.io < 4) ? io_names[k.io] : "?");
    else
        snprintf(buf, n, "k_fft_generic<%d,%s>", k.threads, k.fwd ? "fwd" : "inv");
}

}  // namespace fbfft
